// Graph canonicalisation and the CSR Laplacian (Sec. 2.1: A(p,q) = w(p,q), D(p,p) = sum_t w(p,t),
// L = D - A; Sec. 4: positive weights).
//
// One stable radix sort of the 2m directed entries keyed by (row, column) gives, in order, the
// CSR rows sorted by column with parallel edges adjacent and in input order. Runs of equal keys
// are merged by an FP64 sum rounded once to FP32; the upper-triangle runs, in order, are the
// canonical edge list (edge id = rank among them); a lower-triangle entry finds its edge id by a
// binary search in the mirrored row.
#include <cmath>

#include "sfg_internal.cuh"

namespace {

constexpr int kBlock = 256;

__global__ void k_lap_expand(int32_t n, int64_t m, const int32_t* __restrict__ u,
                             const int32_t* __restrict__ v, const float* __restrict__ w, int bits,
                             uint64_t sent, uint64_t* __restrict__ keys,
                             uint32_t* __restrict__ vals, int* __restrict__ err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = u[e], b = v[e];
        const float ww = w[e];
        const bool bad = a < 0 || a >= n || b < 0 || b >= n || !isfinite(ww) || !(ww > 0.0f);
        if (bad) atomicOr(err, 1);
        uint64_t k0 = sent, k1 = sent;
        if (!bad && a != b) {
            k0 = ((uint64_t)a << bits) | (uint64_t)b;
            k1 = ((uint64_t)b << bits) | (uint64_t)a;
        }
        keys[2 * e] = k0;
        keys[2 * e + 1] = k1;
        vals[2 * e] = (uint32_t)e;
        vals[2 * e + 1] = (uint32_t)e;
    }
}

__global__ void k_lap_heads(const uint64_t* __restrict__ keys, int64_t len, uint64_t sent,
                            uint8_t* __restrict__ head) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        head[i] = (k != sent) && (i == 0 || keys[i - 1] != k);
    }
}

__global__ void k_lap_runs(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                           const float* __restrict__ w, int64_t len, const uint8_t* __restrict__ head,
                           const int64_t* __restrict__ run_off, int bits,
                           int32_t* __restrict__ row_of_run, int2* __restrict__ colval,
                           uint8_t* __restrict__ upper) {
    const uint64_t cmask = (1ull << bits) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!head[i]) continue;
        const uint64_t k = keys[i];
        double s = 0.0;  // parallel edges: FP64 sum in input order, rounded once
        for (int64_t t = i; t < len && keys[t] == k; ++t) s += (double)w[vals[t]];
        const int64_t j = run_off[i];
        const int32_t row = (int32_t)(k >> bits), col = (int32_t)(k & cmask);
        row_of_run[j] = row;
        colval[j] = make_int2(col, __float_as_int((float)s));
        upper[j] = row < col;
    }
}

__global__ void k_lap_rowptr(const int32_t* __restrict__ row_of_run, int64_t nnz, int32_t n,
                             int32_t* __restrict__ row_ptr) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= nnz;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t prev = j > 0 ? row_of_run[j - 1] : -1;
        const int32_t cur = j < nnz ? row_of_run[j] : n;
        for (int32_t r = prev + 1; r <= cur; ++r) row_ptr[r] = (int32_t)j;
    }
}

__global__ void k_lap_upper(const int2* __restrict__ colval, const int32_t* __restrict__ row_of_run,
                            const uint8_t* __restrict__ upper, const int64_t* __restrict__ up_off,
                            int64_t nnz, int32_t* __restrict__ eu, int32_t* __restrict__ ev,
                            float* __restrict__ ew, int32_t* __restrict__ eid) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (!upper[j]) continue;
        const int64_t e = up_off[j];
        const int2 cv = colval[j];
        eu[e] = row_of_run[j];
        ev[e] = cv.x;
        ew[e] = __int_as_float(cv.y);
        eid[j] = (int32_t)e;
    }
}

__global__ void k_lap_lower(const int2* __restrict__ colval, const int32_t* __restrict__ row_of_run,
                            const uint8_t* __restrict__ upper, const int32_t* __restrict__ row_ptr,
                            int64_t nnz, int32_t* __restrict__ eid) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (upper[j]) continue;
        const int32_t r = row_of_run[j], c = colval[j].x;  // entry (r, c), c < r: mirror (c, r)
        int32_t lo = row_ptr[c], hi = row_ptr[c + 1];
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (colval[mid].x < r) lo = mid + 1; else hi = mid;
        }
        eid[j] = eid[lo];
    }
}

__global__ void k_lap_deg(const int32_t* __restrict__ row_ptr, const int2* __restrict__ colval,
                          int32_t n, double* __restrict__ deg, double* __restrict__ invdeg) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;  // in column order
        for (int32_t j = row_ptr[p]; j < row_ptr[p + 1]; ++j) s += (double)__int_as_float(colval[j].y);
        deg[p] = s;
        invdeg[p] = s > 0.0 ? 1.0 / s : 0.0;
    }
}

__global__ void k_lap_f2c(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                          int64_t len, uint64_t sent, const int64_t* __restrict__ run_off,
                          const uint8_t* __restrict__ upper, const int64_t* __restrict__ up_off,
                          int32_t* __restrict__ f2c) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (keys[i] == sent) continue;
        const int64_t j = run_off[i + 1] - 1;  // run holding position i
        if (upper[j]) f2c[vals[i]] = (int32_t)up_off[j];
    }
}

// ---- subgraph ----------------------------------------------------------------------------------
__global__ void k_sub_flags(const int32_t* __restrict__ eid, const uint8_t* __restrict__ mask,
                            int64_t nnz, uint8_t* __restrict__ keep) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x)
        keep[j] = mask[eid[j]] != 0;
}

__global__ void k_mask01(const uint8_t* __restrict__ mask, int64_t m, uint8_t* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = mask[e] != 0;
}

__global__ void k_sub_edges(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                            const float* __restrict__ ew, const uint8_t* __restrict__ keep_e,
                            const int64_t* __restrict__ escan, int64_t m, int32_t* __restrict__ su,
                            int32_t* __restrict__ sv, float* __restrict__ sw) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (!keep_e[e]) continue;
        const int64_t t = escan[e];
        su[t] = eu[e]; sv[t] = ev[e]; sw[t] = ew[e];
    }
}

__global__ void k_sub_csr(const int2* __restrict__ colval, const int32_t* __restrict__ eid,
                          const uint8_t* __restrict__ keep, const int64_t* __restrict__ jscan,
                          const int64_t* __restrict__ escan, int64_t nnz, int2* __restrict__ scv,
                          int32_t* __restrict__ seid) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[j]) continue;
        const int64_t t = jscan[j];
        scv[t] = colval[j];
        seid[t] = (int32_t)escan[eid[j]];
    }
}

__global__ void k_sub_rowptr(const int32_t* __restrict__ row_ptr, const int64_t* __restrict__ jscan,
                             int32_t n, int32_t* __restrict__ srp) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= n;
         p += (int64_t)gridDim.x * blockDim.x)
        srp[p] = (int32_t)jscan[row_ptr[p]];
}

__global__ void k_split_colval(const int2* __restrict__ cv, int64_t nnz, int32_t* __restrict__ col,
                               float* __restrict__ val) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int2 x = cv[j];
        if (col) col[j] = x.x;
        if (val) val[j] = __int_as_float(x.y);
    }
}

int bits_for(int32_t n) {
    int b = 1;
    while (b < 31 && (1ll << b) < (int64_t)n) ++b;
    return b;
}

template <typename K>
int grid_of(sfg_ctx* ctx, K kernel, int64_t work) {
    return sfg_grid(ctx, (const void*)kernel, kBlock, 0, work);
}

}  // namespace

void sfg_graph_free(sfg_graph* g) {
    if (!g) return;
    SfgDeviceGuard guard(g->device);
    cudaStream_t s = g->stream;
    void* ptrs[] = {g->eu, g->ev, g->ew, g->row_ptr, g->colval, g->eid, g->deg, g->invdeg,
                    g->gs_color, g->gs_order, g->hv_rows, g->hv_soff, g->hv_seg, g->gh_rows, g->gh_soff, g->gh_seg};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, s);
    delete g;
}

// Allocate the arrays of a graph with n nodes and m canonical edges.
sfg_status sfg_alloc_graph(sfg_ctx* ctx, int32_t n, int64_t m, sfg_graph** out) {
    sfg_graph* g = new sfg_graph();
    g->device = ctx->device;
    g->n = n;
    g->m = m;
    g->stream = ctx->stream;
    sfg_status st = SFG_OK;
    auto A = [&](void** p, size_t bytes) {
        if (st == SFG_OK) st = sfg_alloc(ctx, p, bytes > 0 ? bytes : 16);
    };
    A((void**)&g->eu, sizeof(int32_t) * m);
    A((void**)&g->ev, sizeof(int32_t) * m);
    A((void**)&g->ew, sizeof(float) * m);
    A((void**)&g->row_ptr, sizeof(int32_t) * ((size_t)n + 1));
    A((void**)&g->colval, sizeof(int2) * 2 * m);
    A((void**)&g->eid, sizeof(int32_t) * 2 * m);
    A((void**)&g->deg, sizeof(double) * n);
    A((void**)&g->invdeg, sizeof(double) * n);
    if (st != SFG_OK) {
        sfg_graph_free(g);
        return st;
    }
    *out = g;
    return SFG_OK;
}

sfg_status sfg_build_graph(sfg_ctx* ctx, int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                           const float* w, bool validate, sfg_graph** out, int32_t* f2c) {
    *out = nullptr;
    const int bits = bits_for(n);
    const uint64_t sent = (bits * 2 >= 64) ? ~0ull : ((1ull << (2 * bits)) - 1);
    const int64_t len = 2 * m;
    Scratch s(ctx);
    uint64_t *keys, *keys2;
    uint32_t *vals, *vals2;
    int* err;
    uint8_t* head;
    int64_t* run_off;
    SFG_TRY(s.get(&keys, len));
    SFG_TRY(s.get(&keys2, len));
    SFG_TRY(s.get(&vals, len));
    SFG_TRY(s.get(&vals2, len));
    SFG_TRY(s.get(&err, 1));
    SFG_TRY(s.get(&head, len));
    SFG_TRY(s.get(&run_off, len + 1));
    SFG_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
    if (m > 0) {
        k_lap_expand<<<grid_of(ctx, k_lap_expand, m), kBlock, 0, ctx->stream>>>(
            n, m, u, v, w, bits, sent, keys, vals, err); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_lap_expand");
    }
    if (validate) {
        int herr = 0;
        SFG_CUDA(ctx, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (herr)
            return sfg_fail(ctx, SFG_EINVAL,
                            "edge list: endpoint outside [0, n) or weight not finite and > 0");
    }
    SFG_TRY(sfg_radix_sort_pairs(ctx, &keys, &vals, &keys2, &vals2, len, 2 * bits));
    int64_t nnz = 0;
    if (len > 0) {
        k_lap_heads<<<grid_of(ctx, k_lap_heads, len), kBlock, 0, ctx->stream>>>(keys, len, sent, head); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_lap_heads");
        SFG_TRY(sfg_scan_u8(ctx, head, run_off, len));
        SFG_TRY(sfg_read_i64(ctx, run_off + len, &nnz));
    }
    if (nnz >= (1ll << 31)) return sfg_fail(ctx, SFG_EINVAL, "too many edges for int32 CSR");
    int32_t* row_of_run;
    int2* colval_tmp;
    uint8_t* upper;
    int64_t* up_off;
    SFG_TRY(s.get(&row_of_run, nnz));
    SFG_TRY(s.get(&colval_tmp, nnz));
    SFG_TRY(s.get(&upper, nnz));
    SFG_TRY(s.get(&up_off, nnz + 1));
    int64_t mc = 0;
    if (nnz > 0) {
        k_lap_runs<<<grid_of(ctx, k_lap_runs, len), kBlock, 0, ctx->stream>>>(
            keys, vals, w, len, head, run_off, bits, row_of_run, colval_tmp, upper); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_lap_runs");
        SFG_TRY(sfg_scan_u8(ctx, upper, up_off, nnz));
        SFG_TRY(sfg_read_i64(ctx, up_off + nnz, &mc));
    }
    sfg_graph* g = nullptr;
    SFG_TRY(sfg_alloc_graph(ctx, n, mc, &g));
    if (nnz > 0)
        SFG_CUDA(ctx, cudaMemcpyAsync(g->colval, colval_tmp, sizeof(int2) * nnz,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    k_lap_rowptr<<<grid_of(ctx, k_lap_rowptr, nnz + 1), kBlock, 0, ctx->stream>>>(row_of_run, nnz,
                                                                                   n, g->row_ptr); ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_lap_rowptr");
    if (nnz > 0) {
        k_lap_upper<<<grid_of(ctx, k_lap_upper, nnz), kBlock, 0, ctx->stream>>>(
            g->colval, row_of_run, upper, up_off, nnz, g->eu, g->ev, g->ew, g->eid); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_lap_upper");
        k_lap_lower<<<grid_of(ctx, k_lap_lower, nnz), kBlock, 0, ctx->stream>>>(
            g->colval, row_of_run, upper, g->row_ptr, nnz, g->eid); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_lap_lower");
    }
    if (n > 0) {
        k_lap_deg<<<grid_of(ctx, k_lap_deg, n), kBlock, 0, ctx->stream>>>(g->row_ptr, g->colval, n,
                                                                          g->deg, g->invdeg); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_lap_deg");
    }
    if (f2c && m > 0) {
        SFG_CUDA(ctx, cudaMemsetAsync(f2c, 0xff, sizeof(int32_t) * m, ctx->stream));
        if (nnz > 0) {
            k_lap_f2c<<<grid_of(ctx, k_lap_f2c, len), kBlock, 0, ctx->stream>>>(
                keys, vals, len, sent, run_off, upper, up_off, f2c); ++ctx->launches;
            SFG_LAUNCH_CHECK(ctx, "k_lap_f2c");
        }
    }
    // the sweep's heavy-row lists are built with the graph, so that later calls (which may be
    // captured into a CUDA graph) never synchronise for them
    const sfg_status hs = sfg_heavy_prepare(ctx, g);
    if (hs != SFG_OK) {
        sfg_graph_free(g);
        return hs;
    }
    *out = g;
    return SFG_OK;
}

sfg_status sfg_subgraph_impl(sfg_ctx* ctx, const sfg_graph* g, const uint8_t* mask,
                             sfg_graph** out) {
    *out = nullptr;
    const int64_t nnz = 2 * g->m;
    Scratch s(ctx);
    uint8_t *keep, *keep_e;
    int64_t *jscan, *escan;
    SFG_TRY(s.get(&keep, nnz));
    SFG_TRY(s.get(&keep_e, g->m));
    SFG_TRY(s.get(&jscan, nnz + 1));
    SFG_TRY(s.get(&escan, g->m + 1));
    int64_t ms = 0;
    if (g->m > 0) {
        k_mask01<<<grid_of(ctx, k_mask01, g->m), kBlock, 0, ctx->stream>>>(mask, g->m, keep_e); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_mask01");
        k_sub_flags<<<grid_of(ctx, k_sub_flags, nnz), kBlock, 0, ctx->stream>>>(g->eid, mask, nnz,
                                                                                keep); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_sub_flags");
        SFG_TRY(sfg_scan_u8(ctx, keep_e, escan, g->m));
        SFG_TRY(sfg_scan_u8(ctx, keep, jscan, nnz));
        SFG_TRY(sfg_read_i64(ctx, escan + g->m, &ms));
    } else {
        SFG_CUDA(ctx, cudaMemsetAsync(jscan, 0, sizeof(int64_t), ctx->stream));
    }
    sfg_graph* p = nullptr;
    SFG_TRY(sfg_alloc_graph(ctx, g->n, ms, &p));
    if (g->m > 0) {
        k_sub_edges<<<grid_of(ctx, k_sub_edges, g->m), kBlock, 0, ctx->stream>>>(
            g->eu, g->ev, g->ew, keep_e, escan, g->m, p->eu, p->ev, p->ew); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_sub_edges");
        k_sub_csr<<<grid_of(ctx, k_sub_csr, nnz), kBlock, 0, ctx->stream>>>(
            g->colval, g->eid, keep, jscan, escan, nnz, p->colval, p->eid); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_sub_csr");
    }
    k_sub_rowptr<<<grid_of(ctx, k_sub_rowptr, (int64_t)g->n + 1), kBlock, 0, ctx->stream>>>(
        g->row_ptr, jscan, g->n, p->row_ptr); ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_sub_rowptr");
    if (g->n > 0) {
        k_lap_deg<<<grid_of(ctx, k_lap_deg, g->n), kBlock, 0, ctx->stream>>>(p->row_ptr, p->colval,
                                                                             g->n, p->deg, p->invdeg); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_lap_deg");
    }
    const sfg_status hs = sfg_heavy_prepare(ctx, p);
    if (hs != SFG_OK) {
        sfg_graph_free(p);
        return hs;
    }
    *out = p;
    return SFG_OK;
}

extern "C" {

sfg_status sfg_laplacian(sfg_ctx* ctx, int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                         const float* w, sfg_graph** out) {
    if (!ctx || !out) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    *out = nullptr;
    if (n < 1) return sfg_fail(ctx, SFG_EINVAL, "n must be >= 1 (got %d)", n);
    if (m < 0 || m >= (1ll << 31)) return sfg_fail(ctx, SFG_EINVAL, "m out of range");
    if (m > 0) {
        SFG_TRY(sfg_check_dev(ctx, u, "u"));
        SFG_TRY(sfg_check_dev(ctx, v, "v"));
        SFG_TRY(sfg_check_dev(ctx, w, "w"));
    }
    return sfg_build_graph(ctx, n, m, u, v, w, true, out, nullptr);
}

void sfg_graph_destroy(sfg_graph* g) { sfg_graph_free(g); }

sfg_status sfg_graph_info(const sfg_graph* g, int32_t* n_host, int64_t* m_host) {
    if (!g) return SFG_EINVAL;
    if (n_host) *n_host = g->n;
    if (m_host) *m_host = g->m;
    return SFG_OK;
}

sfg_status sfg_graph_edges(sfg_ctx* ctx, const sfg_graph* g, int32_t* u, int32_t* v, float* w) {
    if (!ctx || !g) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (g->m == 0) return SFG_OK;
    if (u) SFG_CUDA(ctx, cudaMemcpyAsync(u, g->eu, 4 * g->m, cudaMemcpyDeviceToDevice, ctx->stream));
    if (v) SFG_CUDA(ctx, cudaMemcpyAsync(v, g->ev, 4 * g->m, cudaMemcpyDeviceToDevice, ctx->stream));
    if (w) SFG_CUDA(ctx, cudaMemcpyAsync(w, g->ew, 4 * g->m, cudaMemcpyDeviceToDevice, ctx->stream));
    return SFG_OK;
}

sfg_status sfg_graph_csr(sfg_ctx* ctx, const sfg_graph* g, int32_t* row_ptr, int32_t* col,
                         float* val, int32_t* eid, double* deg) {
    if (!ctx || !g) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    const int64_t nnz = 2 * g->m;
    if (row_ptr)
        SFG_CUDA(ctx, cudaMemcpyAsync(row_ptr, g->row_ptr, 4 * ((size_t)g->n + 1),
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    if (deg)
        SFG_CUDA(ctx, cudaMemcpyAsync(deg, g->deg, 8 * (size_t)g->n, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
    if (nnz == 0) return SFG_OK;
    if (eid)
        SFG_CUDA(ctx, cudaMemcpyAsync(eid, g->eid, 4 * nnz, cudaMemcpyDeviceToDevice, ctx->stream));
    if (col || val) {
        k_split_colval<<<grid_of(ctx, k_split_colval, nnz), kBlock, 0, ctx->stream>>>(g->colval, nnz,
                                                                                      col, val); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_split_colval");
    }
    return SFG_OK;
}

sfg_status sfg_graph_subgraph(sfg_ctx* ctx, const sfg_graph* g, const uint8_t* mask,
                              sfg_graph** out) {
    if (!ctx || !g || !out) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    *out = nullptr;
    if (g->m > 0) SFG_TRY(sfg_check_dev(ctx, mask, "mask"));
    return sfg_subgraph_impl(ctx, g, mask, out);
}

}  // extern "C"
