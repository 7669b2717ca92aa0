// Context, status, allocation and timing plumbing of libsfg.
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "sfg_internal.cuh"

sfg_status sfg_fail(sfg_ctx* ctx, sfg_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return st;
}

sfg_status sfg_cuda_fail(sfg_ctx* ctx, cudaError_t e, const char* where) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return sfg_fail(ctx, SFG_ENOMEM, "out of device memory in %s", where);
    }
    return sfg_fail(ctx, SFG_ECUDA, "CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e),
                    where);
}

sfg_status sfg_alloc(sfg_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    ctx->alloc_count++;
    if (ctx->fail_alloc_at >= 0 && ctx->alloc_count == ctx->fail_alloc_at)
        return sfg_fail(ctx, SFG_ENOMEM, "injected allocation failure (allocation %lld)",
                        (long long)ctx->alloc_count);
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream);
    if (e == cudaErrorMemoryAllocation) {
        // the pool keeps freed memory; hand it back to the device and try once more
        cudaGetLastError();
        cudaStreamSynchronize(ctx->stream);
        cudaMemPoolTrimTo(ctx->pool, 0);
        e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return sfg_fail(ctx, SFG_ENOMEM, "cudaMallocFromPoolAsync(%zu bytes) failed: %s", bytes,
                        cudaGetErrorString(e));
    }
    return SFG_OK;
}

void sfg_free(sfg_ctx* ctx, void* p) {
    if (p) cudaFreeAsync(p, ctx->stream);
}

sfg_status sfg_host_word(sfg_ctx* ctx, int slot, int** out) {
    if (!ctx->host_word)
        SFG_CUDA(ctx, cudaMallocHost((void**)&ctx->host_word, sizeof(int) * kSfgHostWords));
    *out = ctx->host_word + slot;
    return SFG_OK;
}

sfg_status sfg_check_dev(sfg_ctx* ctx, const void* p, const char* what) {
    if (!p) return sfg_fail(ctx, SFG_EINVAL, "%s is NULL", what);
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfg_fail(ctx, SFG_EINVAL, "%s is not a CUDA pointer", what);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return sfg_fail(ctx, SFG_EINVAL, "%s is not device memory", what);
    return SFG_OK;
}

int sfg_grid(sfg_ctx* ctx, const void* kernel, int block, size_t smem, int64_t work_items) {
    // resident CTAs per SM, asked once per (kernel, block, shared memory) and context
    const auto key = std::make_tuple(kernel, block, smem);
    auto it = ctx->occupancy.find(key);
    int per_sm = 0;
    if (it != ctx->occupancy.end()) {
        per_sm = it->second;
    } else {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        ctx->occupancy.emplace(key, per_sm);
    }
    int64_t full = (int64_t)per_sm * ctx->num_sms;
    int64_t need = (work_items + block - 1) / block;
    if (need < 1) need = 1;
    return (int)(need < full ? need : full);
}

void sfg_tic(sfg_ctx* ctx, const char* name) {
    if (!ctx->timing) return;
    sfg_timer_rec r;
    r.name = name;
    for (int i = 0; i < 2; ++i) {
        cudaEvent_t ev;
        if (!ctx->event_pool.empty()) {
            ev = ctx->event_pool.back();
            ctx->event_pool.pop_back();
        } else if (cudaEventCreate(&ev) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        (i == 0 ? r.start : r.stop) = ev;
    }
    cudaEventRecord(r.start, ctx->stream);
    ctx->timers.push_back(r);
}

void sfg_toc(sfg_ctx* ctx) {
    if (!ctx->timing || ctx->timers.empty()) return;
    cudaEventRecord(ctx->timers.back().stop, ctx->stream);
}

uint32_t sfg_tune_key(int K, sfg_dtype dt, int bucket) {
    return ((uint32_t)K << 16) | ((uint32_t)dt << 8) | (uint32_t)bucket;
}

int sfg_degree_bucket(const sfg_graph* L) {
    const double avg = L->n > 0 ? (2.0 * (double)L->m) / (double)L->n : 0.0;
    int b = 0;
    while (b < 15 && (double)(2 << b) <= avg) ++b;  // bucket b: 2^b <= avg degree < 2^(b+1)
    return b;
}

int sfg_tuned_variant(const sfg_ctx* ctx, int K, sfg_dtype dt, const sfg_graph* L) {
    if (ctx->tune.empty()) return -1;
    auto it = ctx->tune.find(sfg_tune_key(K, dt, sfg_degree_bucket(L)));
    return it == ctx->tune.end() ? -1 : it->second;
}

void sfg_tune_record(sfg_ctx* ctx, int K, sfg_dtype dt, const sfg_graph* L, int variant) {
    ctx->tune[sfg_tune_key(K, dt, sfg_degree_bucket(L))] = variant;
}

int sfg_score_shape(const sfg_ctx* ctx, int K, sfg_dtype dt, const sfg_graph* L) {
    const int b = sfg_degree_bucket(L);
    if (!ctx->score_tune.empty()) {
        auto it = ctx->score_tune.find(sfg_tune_key(K, dt, b));
        if (it != ctx->score_tune.end()) return it->second;
    }
    return b <= 2 ? 0 : 1;
}

extern "C" {

// The library's memory pool on `device`: created on first use and kept for the life of the
// process, shared by every context on the device, with a release threshold that keeps freed
// memory mapped (the device's default pool returns everything at each synchronisation, and the
// next large block then pays for mapping it again). Graphs and networks may outlive the context
// that made them, so the pool is never destroyed; contexts only trim it.
static cudaMemPool_t device_pool(int device) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lock(mu);
    auto it = pools.find(device);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps pp = {};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &pp) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[device] = pool;
    return pool;
}

sfg_status sfg_ctx_create(sfg_ctx** out, int device, void* cuda_stream) {
    if (!out) return SFG_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return SFG_EINVAL;
    }
    SfgDeviceGuard guard(device);
    sfg_ctx* c = new sfg_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (c->num_sms < 1) c->num_sms = 1;
    if (const char* f = std::getenv("SFG_FAULT_ALLOC")) c->fail_alloc_at = std::atoll(f);
    if (const char* f = std::getenv("SFG_FAULT_MMA_WAIT")) c->withhold_mma = std::atoi(f) != 0;
    c->pool = device_pool(device);
    if (!c->pool) {
        delete c;
        return SFG_ECUDA;
    }
    // The allocation-free entry points' file-scope scratch is resolved here, so that the module
    // that holds it is loaded (and its memory taken) when a context is created, never inside
    // one of those calls.
    if (sfg_noalloc_prepare(c) != SFG_OK) {
        delete c;
        return SFG_ECUDA;
    }
    *out = c;
    return SFG_OK;
}

sfg_status sfg_ctx_trim(sfg_ctx* ctx) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    SFG_CUDA(ctx, cudaMemPoolTrimTo(ctx->pool, 0));
    return SFG_OK;
}

void sfg_ctx_destroy(sfg_ctx* ctx) {
    if (!ctx) return;
    SFG_DEVICE(ctx);
    for (auto& r : ctx->timers) {
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->host_word) {
        cudaStreamSynchronize(ctx->stream);
        cudaFreeHost(ctx->host_word);
    }
    if (ctx->pool) {
        // unused memory goes back to the device; memory of live graphs stays valid
        cudaStreamSynchronize(ctx->stream);
        cudaMemPoolTrimTo(ctx->pool, 0);
    }
    delete ctx;
}

sfg_status sfg_ctx_set_stream(sfg_ctx* ctx, void* cuda_stream) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    ctx->stream = (cudaStream_t)cuda_stream;
    return SFG_OK;
}

const char* sfg_last_error(const sfg_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

sfg_status sfg_ctx_timing(sfg_ctx* ctx, int on) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (auto& r : ctx->timers) {
        ctx->event_pool.push_back(r.start);
        ctx->event_pool.push_back(r.stop);
    }
    ctx->timers.clear();
    ctx->timing = on != 0;
    return SFG_OK;
}

sfg_status sfg_ctx_kernel_time(sfg_ctx* ctx, const char* prefix, int64_t* launches_host,
                               double* ms_host) {
    if (!ctx || !prefix || !launches_host || !ms_host) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int64_t n = 0;
    double total = 0.0;
    size_t len = std::strlen(prefix);
    for (auto& r : ctx->timers) {
        if (std::strncmp(r.name, prefix, len) != 0) continue;
        float ms = 0.f;
        SFG_CUDA(ctx, cudaEventElapsedTime(&ms, r.start, r.stop));
        total += ms;
        ++n;
    }
    *launches_host = n;
    *ms_host = total;
    return SFG_OK;
}

sfg_status sfg_ctx_launches(const sfg_ctx* ctx, int64_t* launches_host) {
    if (!ctx || !launches_host) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    *launches_host = ctx->launches;
    return SFG_OK;
}

sfg_status sfg_autotune(sfg_ctx* ctx, const sfg_graph* L, int K, sfg_dtype storage,
                        int* variant_host, double* us_per_sweep_host) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!L) return sfg_fail(ctx, SFG_EINVAL, "graph is NULL");
    if (!sfg_k_supported(K, storage))
        return sfg_fail(ctx, SFG_EUNSUPPORTED, "K=%d unsupported for dtype %d", K, (int)storage);
    return sfg_autotune_impl(ctx, L, K, storage, variant_host, us_per_sweep_host);
}

sfg_status sfg_tune_set(sfg_ctx* ctx, int K, sfg_dtype storage, int degree_bucket, int variant) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (degree_bucket < 0 || degree_bucket > 15 || variant < -1 || variant >= SFG_SWEEP_VARIANTS)
        return sfg_fail(ctx, SFG_EINVAL, "bad tuning entry");
    const uint32_t key = sfg_tune_key(K, storage, degree_bucket);
    if (variant < 0) ctx->tune.erase(key);
    else ctx->tune[key] = variant;
    return SFG_OK;
}

sfg_status sfg_tune_set_score(sfg_ctx* ctx, int K, sfg_dtype storage, int degree_bucket,
                              int shape) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (degree_bucket < 0 || degree_bucket > 15 || shape < -1 || shape >= SFG_SCORE_SHAPES)
        return sfg_fail(ctx, SFG_EINVAL, "bad tuning entry");
    const uint32_t key = sfg_tune_key(K, storage, degree_bucket);
    if (shape < 0) ctx->score_tune.erase(key);
    else ctx->score_tune[key] = shape;
    return SFG_OK;
}

sfg_status sfg_tune_table(const sfg_ctx* ctx, char* buf, int64_t cap, int64_t* len_host) {
    if (!ctx || !len_host) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    static const int tpi[SFG_SWEEP_VARIANTS] = {1, 2, 4, 1, 2, 4};
    static const int minb[SFG_SWEEP_VARIANTS] = {4, 4, 4, 3, 3, 3};
    std::map<uint32_t, std::pair<int, int>> keys;  // key -> (sweep variant, scorer shape)
    for (auto& kv : ctx->tune) keys[kv.first] = {kv.second, -1};
    for (auto& kv : ctx->score_tune) {
        auto it = keys.find(kv.first);
        if (it == keys.end()) keys[kv.first] = {-1, kv.second};
        else it->second.second = kv.second;
    }
    std::string j = "[";
    for (auto& kv : keys) {
        char item[224];
        const int v = kv.second.first, s = kv.second.second;
        snprintf(item, sizeof item,
                 "%s{\"K\": %u, \"dtype\": %u, \"degree_bucket\": %u, \"variant\": %d, "
                 "\"tiles_per_warp\": %d, \"ctas_per_sm\": %d, \"score_shape\": %d}",
                 j.size() > 1 ? ", " : "", kv.first >> 16, (kv.first >> 8) & 0xff, kv.first & 0xff,
                 v, v >= 0 ? tpi[v] : 0, v >= 0 ? minb[v] : 0, s);
        j += item;
    }
    j += "]";
    *len_host = (int64_t)j.size();
    if (buf && cap > 0) {
        const size_t n = std::min((size_t)cap - 1, j.size());
        memcpy(buf, j.data(), n);
        buf[n] = 0;
        if ((int64_t)j.size() >= cap) return SFG_ECAPACITY;
    }
    return SFG_OK;
}

}  // extern "C"
