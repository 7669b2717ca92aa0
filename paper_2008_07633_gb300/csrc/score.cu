// Edge scores. (1) Spectral-perturbation score of candidate edges (Sec. 3.5, Eqs.
// formula_eig_perturb1_conclusion / formula_eig_perturb1_conclusion2 with U replaced by the
// smoothed blocks; the scoring and selection steps of Algorithm 1). (2) Algebraic-distance affinity that drives node
// aggregation in coarsening (Sec. 3.2).
//
// Scorer schedule: one LPR-lane group per listed edge; the group gathers the two endpoint rows of
// both blocks (one 32-byte load per row and lane), forms the two squared distances in FP32 and
// folds them with xor-shuffles inside the group.
#include "sfg_internal.cuh"
#include "vec.cuh"

namespace {

constexpr int kBlock = 256;

// One 32-byte global load (sm_100 and later) into two 16-byte vectors; p must be 32-byte aligned.
template <int CG>
__device__ __forceinline__ void load_raw32(const void* p, uint4& a, uint4& b) {
    if (CG)  // cached in L2 only
        asm volatile("ld.global.cg.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                     : "l"(p));
    else
        asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                     : "l"(p));
}

// One 16-byte row vector; CG: cached in L2 only.
template <typename T, int CG>
__device__ __forceinline__ uint4 load_row16(const T* p) {
    if (!CG) return Vec<T>::load_raw(p);
    uint4 r;
    asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}

template <int LPR>
__device__ __forceinline__ unsigned group_mask(int lane) {
    if (LPR == 32) return 0xffffffffu;
    return ((1u << LPR) - 1u) << ((lane / LPR) * LPR);
}

// Scorer, warp-tile schedule: a warp scores U consecutive tiles of GPW = 32 / LPR list entries
// each (one LPR-lane group per edge) and moves by grid stride over such tile groups. Lane s of a
// group holds V consecutive 16-byte vectors of a row (entries [s V E, (s + 1) V E)); with V = 2 a
// row is read by one 32-byte load per lane when both blocks are 32-byte aligned (WIDE, the usual
// case) and by two 16-byte loads otherwise, with the same arithmetic. Every lane of a group
// loads its edge's id, endpoints and weight itself (group-uniform addresses are served as one
// broadcast). The next group's endpoints and the ids of the group after it are loaded before this
// group's 4U row gathers are consumed, so one gather round is the exposed latency per U tiles;
// gathered rows stay packed until they are used. The two squared distances are folded together:
// at the first step the even lane of each pair keeps the G partial and the odd lane the P partial,
// so one shuffle per level moves both, and one more hands the P sum to the group's first lane.
// The score formula is fixed at compile time (MODE); U, MINB (CTAs per SM) and CG (row loads
// cached in L2 only, not in L1) are the launch shape.
// SCALED: the blocks are raw smoothed blocks and column k of each is multiplied by its projection
// scale (sg, sp) on the fly; the projection's mean removal cancels in X_p - X_q.
// SCALED = 2: the scales are per graph of a disjoint union (graph g's rows start at node_off[g]),
// looked up from each edge's first endpoint.
template <typename T, int LPR, int V, bool WIDE, int SCALED, int U, int MINB, int CG, int MODE>
__global__ void __launch_bounds__(kBlock, MINB)
    k_score(int64_t ne, const int32_t* __restrict__ ids, const int32_t* __restrict__ eu,
             const int32_t* __restrict__ ev, const float* __restrict__ ew,
             const T* __restrict__ XG, const T* __restrict__ XP, float eta,
             const float* __restrict__ sg, const float* __restrict__ sp,
             const int32_t* __restrict__ node_off, int ngraphs, float* __restrict__ out) {
    static_assert(V == 1 || V == 2, "one or two vectors per lane");
    constexpr int E = Vec<T>::E, K = LPR * E * V, GPW = 32 / LPR;
    const int lane = threadIdx.x & 31, grp = lane / LPR, sub = lane % LPR;
    const unsigned gm = group_mask<LPR>(lane);
    const int64_t wid = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int64_t nw = (int64_t)gridDim.x * (kBlock / 32);
    const int64_t ntiles = (ne + GPW - 1) / GPW;
    const int64_t ngroups = (ntiles + U - 1) / U;
    const int sub0 = sub * V * E;  // first entry of this lane
    const T* __restrict__ Xg = XG + sub0;
    const T* __restrict__ Xp = XP + sub0;
    __shared__ float s_scale[2][SCALED == 1 ? K : 1];
    if (SCALED == 1) {
        for (int k = threadIdx.x; k < K; k += kBlock) {
            s_scale[0][k] = sg[k];
            s_scale[1][k] = sp[k];
        }
        __syncthreads();
    }
    // this group's list entry in tile t (-1 past the end)
    auto load_id = [&](int64_t t) -> int32_t {
        const int64_t i = t * GPW + grp;
        return i < ne ? ids[i] : -1;
    };
    struct Edge { int32_t p, q; float w; };
    auto load_edge = [&](int32_t e) {
        Edge d{0, 0, 0.f};
        if (e >= 0) { d.p = eu[e]; d.q = ev[e]; d.w = ew[e]; }
        return d;
    };
    int64_t g = wid;
    Edge cur[U];
    int32_t idn[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        cur[u] = load_edge(load_id(g * U + u));
        idn[u] = load_id((g + nw) * U + u);
    }
    for (; g < ngroups; g += nw) {
        Edge nxt[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            nxt[u] = load_edge(idn[u]);
            idn[u] = load_id((g + 2 * nw) * U + u);
        }
        uint4 rgp[U][V], rgq[U][V], rpp[U][V], rpq[U][V];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t p = cur[u].p, q = cur[u].q;
            if constexpr (V == 2 && WIDE) {
                load_raw32<CG>(Xg + p * K, rgp[u][0], rgp[u][V - 1]);
                load_raw32<CG>(Xg + q * K, rgq[u][0], rgq[u][V - 1]);
                load_raw32<CG>(Xp + p * K, rpp[u][0], rpp[u][V - 1]);
                load_raw32<CG>(Xp + q * K, rpq[u][0], rpq[u][V - 1]);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    rgp[u][v] = load_row16<T, CG>(Xg + p * K + v * E);
                    rgq[u][v] = load_row16<T, CG>(Xg + q * K + v * E);
                    rpp[u][v] = load_row16<T, CG>(Xp + p * K + v * E);
                    rpq[u][v] = load_row16<T, CG>(Xp + q * K + v * E);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = (g * U + u) * GPW + grp;
            const float* sc_g = nullptr;
            const float* sc_p = nullptr;
            if (SCALED == 1) {
                sc_g = s_scale[0] + sub0;
                sc_p = s_scale[1] + sub0;
            } else if (SCALED == 2) {
                const int32_t p = cur[u].p;
                int lo = 0, hi = ngraphs;  // graph of row p
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (node_off[mid] <= p) lo = mid; else hi = mid;
                }
                sc_g = sg + (size_t)lo * K + sub0;
                sc_p = sp + (size_t)lo * K + sub0;
            }
            float dg = 0.f, dp = 0.f;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                float gp[E], gq[E], pp[E], pq[E];
                Vec<T>::unpack(rgp[u][v], gp);
                Vec<T>::unpack(rgq[u][v], gq);
                Vec<T>::unpack(rpp[u][v], pp);
                Vec<T>::unpack(rpq[u][v], pq);
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    float a = gp[k] - gq[k], b = pp[k] - pq[k];
                    if (SCALED) {
                        a *= sc_g[v * E + k];
                        b *= sc_p[v * E + k];
                    }
                    dg = fmaf(a, a, dg);
                    dp = fmaf(b, b, dp);
                }
            }
            if (LPR > 1) {
                // even lanes: G partial sums, odd lanes: P partial sums
                const bool odd = sub & 1;
                const float give = odd ? dg : dp;
                const float got = __shfl_xor_sync(gm, give, 1, LPR);
                float v = (odd ? dp : dg) + got;
#pragma unroll
                for (int o = 2; o < LPR; o <<= 1) v += __shfl_xor_sync(gm, v, o, LPR);
                const float other = __shfl_xor_sync(gm, v, 1, LPR);
                dg = v;
                dp = other;
            }
            if (sub == 0 && i < ne) {
                const float w = cur[u].w;
                const float sgv = w * dg, spv = w * dp;
                out[i] = MODE == SFG_SCORE_G ? sgv : (MODE == SFG_SCORE_P ? spv : spv / (sgv + eta));
            }
            cur[u] = nxt[u];
        }
    }
}

// Stored block entry widened to FP64 (exact for FP32 and BF16).
__device__ __forceinline__ double widen(float x) { return (double)x; }
__device__ __forceinline__ double widen(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

// ||X_p||^2 in FP64, increasing k, no fused multiply-add.
template <typename T>
__global__ void k_rownorm(int32_t n, const T* __restrict__ X, int K, double* __restrict__ nn) {
    for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kBlock) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) {
            const double x = widen(X[p * K + k]);
            s = __dadd_rn(s, __dmul_rn(x, x));
        }
        nn[p] = s;
    }
}

// delta_e = 1 - (X_p . X_q)^2 / (||X_p||^2 ||X_q||^2) in FP64, same operation order as the
// definition, no fused multiply-add; a zero row gives 1.
template <typename T>
__global__ void k_affinity(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                           const T* __restrict__ X, int K, const double* __restrict__ nn,
                           double* __restrict__ delta) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock) {
        const int64_t p = eu[e], q = ev[e];
        double dot = 0.0;
        for (int k = 0; k < K; ++k)
            dot = __dadd_rn(dot, __dmul_rn(widen(X[p * K + k]), widen(X[q * K + k])));
        const double den = __dmul_rn(nn[p], nn[q]);
        delta[e] = den > 0.0 ? __dsub_rn(1.0, __ddiv_rn(__dmul_rn(dot, dot), den)) : 1.0;
    }
}

// NV: 16-byte vectors per row; each lane takes two of them (one when a row is one vector).
// Launch shape 0: one tile per warp iteration, four CTAs per SM; shape 1: two tiles, two CTAs per
// SM; shape 2: shape 0 with row loads cached in L2 only (sfg_score_shape). All compute the same
// values bit for bit.
template <typename T, int NV>
sfg_status launch_score(sfg_ctx* ctx, const sfg_graph* LG, const void* XG, const void* XP,
                        const int32_t* ids, int64_t ne, int mode, const float* sg,
                        const float* sp, const int32_t* node_off, int ngraphs, float* out) {
    if (ne == 0) return SFG_OK;
    constexpr int V = NV >= 2 ? 2 : 1, LPR = NV / V;
    constexpr int K = NV * 16 / (int)sizeof(T);
    const T *xg = (const T*)XG, *xp = (const T*)XP;
    float eta = 1e-30f;
    const bool wide = V == 2 && ((((uintptr_t)XG | (uintptr_t)XP) & 31) == 0);
    const int sc = node_off ? 2 : (sg ? 1 : 0);
    const int shape = sfg_score_shape(ctx, K, sizeof(T) == 2 ? SFG_BF16 : SFG_F32, LG);
    constexpr bool W2 = V == 2;  // 32-byte loads exist only for two vectors per lane
#define SFG_SCORE_ROW(WD, SC, U, MB, CG)                                                            \
    {(void*)k_score<T, LPR, V, WD, SC, U, MB, CG, 0>, (void*)k_score<T, LPR, V, WD, SC, U, MB, CG, 1>, \
     (void*)k_score<T, LPR, V, WD, SC, U, MB, CG, 2>}
#define SFG_SCORE_SHAPE(WD, U, MB, CG)                                                              \
    {SFG_SCORE_ROW(WD, 0, U, MB, CG), SFG_SCORE_ROW(WD, 1, U, MB, CG), SFG_SCORE_ROW(WD, 2, U, MB, CG)}
    static void* const tab[2][SFG_SCORE_SHAPES][3][3] = {
        {SFG_SCORE_SHAPE(false, 1, 4, 0), SFG_SCORE_SHAPE(false, 2, 2, 0), SFG_SCORE_SHAPE(false, 1, 4, 1)},
        {SFG_SCORE_SHAPE(W2, 1, 4, 0), SFG_SCORE_SHAPE(W2, 2, 2, 0), SFG_SCORE_SHAPE(W2, 1, 4, 1)}};
#undef SFG_SCORE_SHAPE
#undef SFG_SCORE_ROW
    const void* k = tab[wide][shape][sc][mode];
    const int U = shape == 1 ? 2 : 1;
    void* args[] = {(void*)&ne, (void*)&ids, (void*)&LG->eu, (void*)&LG->ev, (void*)&LG->ew,
                    (void*)&xg, (void*)&xp, (void*)&eta, (void*)&sg, (void*)&sp,
                    (void*)&node_off, (void*)&ngraphs, (void*)&out};
    const int grid = sfg_grid(ctx, k, kBlock, 0, (ne + U - 1) / U * LPR);
    sfg_tic(ctx, "score");
    const cudaError_t e = cudaLaunchKernel(k, dim3(grid), dim3(kBlock), args, 0, ctx->stream);
    if (e != cudaSuccess) return sfg_cuda_fail(ctx, e, "k_score");
    ++ctx->launches;
    sfg_toc(ctx);
    SFG_LAUNCH_CHECK(ctx, "k_score");
    return SFG_OK;
}

}  // namespace

sfg_status sfg_score_batched_impl(sfg_ctx* ctx, const sfg_graph* LG, const void* XG,
                                  const void* XP, int K, sfg_dtype storage, const int32_t* ids,
                                  int64_t ne, sfg_score_mode mode, float* out, const float* sg,
                                  const float* sp, const int32_t* node_off, int ngraphs) {
#define SFG_SCORE_CASE(TY, L) \
    return launch_score<TY, L>(ctx, LG, XG, XP, ids, ne, mode, sg, sp, node_off, ngraphs, out)
    if (storage == SFG_F32) {
        switch (K) {
            case 4: SFG_SCORE_CASE(float, 1);
            case 8: SFG_SCORE_CASE(float, 2);
            case 16: SFG_SCORE_CASE(float, 4);
            case 32: SFG_SCORE_CASE(float, 8);
            case 64: SFG_SCORE_CASE(float, 16);
        }
    } else if (storage == SFG_BF16) {
        switch (K) {
            case 8: SFG_SCORE_CASE(__nv_bfloat16, 1);
            case 16: SFG_SCORE_CASE(__nv_bfloat16, 2);
            case 32: SFG_SCORE_CASE(__nv_bfloat16, 4);
            case 64: SFG_SCORE_CASE(__nv_bfloat16, 8);
        }
    }
#undef SFG_SCORE_CASE
    return sfg_fail(ctx, SFG_EUNSUPPORTED, "K=%d unsupported for dtype %d", K, (int)storage);
}

namespace {
__global__ void k_iota(int64_t m, int32_t* __restrict__ ids) {
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < m; i += (int64_t)gridDim.x * kBlock)
        ids[i] = (int32_t)i;
}
}  // namespace

sfg_status sfg_score_autotune_impl(sfg_ctx* ctx, const sfg_graph* L, int K, sfg_dtype storage,
                                   const void* X) {
    if (L->m == 0) return SFG_OK;
    Scratch s(ctx);
    int32_t* ids;
    float* out;
    SFG_TRY(s.get(&ids, (size_t)L->m));
    SFG_TRY(s.get(&out, (size_t)L->m));
    k_iota<<<sfg_grid(ctx, (const void*)k_iota, kBlock, 0, L->m), kBlock, 0, ctx->stream>>>(L->m, ids);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_iota");
    const uint32_t key = sfg_tune_key(K, storage, sfg_degree_bucket(L));
    const auto it0 = ctx->score_tune.find(key);
    const int saved = it0 == ctx->score_tune.end() ? -1 : it0->second;
    cudaEvent_t e0, e1;
    SFG_CUDA(ctx, cudaEventCreate(&e0));
    SFG_CUDA(ctx, cudaEventCreate(&e1));
    int best = 0;
    float best_ms = 1e30f;
    sfg_status st = SFG_OK;
    for (int shape = 0; shape < SFG_SCORE_SHAPES && st == SFG_OK; ++shape) {
        ctx->score_tune[key] = shape;
        for (int r = 0; r < 4 && st == SFG_OK; ++r) {  // one warm-up, three timed
            if (r == 1) cudaEventRecord(e0, ctx->stream);
            st = sfg_score_impl(ctx, L, X, X, K, storage, ids, L->m, SFG_SCORE_RATIO, out, nullptr,
                                nullptr);
        }
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = shape; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SFG_OK) {
        if (saved < 0) ctx->score_tune.erase(key);
        else ctx->score_tune[key] = saved;
        return st;
    }
    ctx->score_tune[key] = best;
    return SFG_OK;
}

sfg_status sfg_score_impl(sfg_ctx* ctx, const sfg_graph* LG, const void* XG, const void* XP,
                          int K, sfg_dtype storage, const int32_t* ids, int64_t ne,
                          sfg_score_mode mode, float* out, const float* sg, const float* sp) {
    return sfg_score_batched_impl(ctx, LG, XG, XP, K, storage, ids, ne, mode, out, sg, sp, nullptr,
                                  0);
}

namespace {
template <typename T>
sfg_status affinity_t(sfg_ctx* ctx, const sfg_graph* L, const T* X, int K, double* delta) {
    Scratch s(ctx);
    double* nn;
    SFG_TRY(s.get(&nn, (size_t)L->n));
    k_rownorm<T><<<sfg_grid(ctx, (const void*)k_rownorm<T>, kBlock, 0, L->n), kBlock, 0,
                   ctx->stream>>>(L->n, X, K, nn);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_rownorm");
    if (L->m > 0) {
        sfg_tic(ctx, "affinity");
        k_affinity<T><<<sfg_grid(ctx, (const void*)k_affinity<T>, kBlock, 0, L->m), kBlock, 0,
                        ctx->stream>>>(L->m, L->eu, L->ev, X, K, nn, delta);
        ++ctx->launches;
        sfg_toc(ctx);
        SFG_LAUNCH_CHECK(ctx, "k_affinity");
    }
    return SFG_OK;
}
}  // namespace

sfg_status sfg_affinity_impl(sfg_ctx* ctx, const sfg_graph* L, const void* X, int K,
                             sfg_dtype storage, double* delta) {
    if (storage == SFG_BF16)
        return affinity_t(ctx, L, (const __nv_bfloat16*)X, K, delta);
    return affinity_t(ctx, L, (const float*)X, K, delta);
}

extern "C" {

sfg_status sfg_score_edges(sfg_ctx* ctx, const sfg_graph* LG, const void* XG, const void* XP,
                           int K, sfg_dtype storage, const int32_t* edge_ids, int64_t ne,
                           sfg_score_mode mode, float* scores_out) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!LG) return sfg_fail(ctx, SFG_EINVAL, "graph is NULL");
    if (ne < 0) return sfg_fail(ctx, SFG_EINVAL, "ne must be >= 0");
    if (mode != SFG_SCORE_RATIO && mode != SFG_SCORE_G && mode != SFG_SCORE_P)
        return sfg_fail(ctx, SFG_EINVAL, "unknown score mode %d", (int)mode);
    if (!sfg_k_supported(K, storage))
        return sfg_fail(ctx, SFG_EUNSUPPORTED, "K=%d unsupported for dtype %d", K, (int)storage);
    if (ne == 0) return SFG_OK;
    SFG_TRY(sfg_check_dev(ctx, XG, "XG"));
    SFG_TRY(sfg_check_dev(ctx, XP, "XP"));
    SFG_TRY(sfg_check_dev(ctx, edge_ids, "edge_ids"));
    SFG_TRY(sfg_check_dev(ctx, scores_out, "scores_out"));
    if ((((uintptr_t)XG) | ((uintptr_t)XP)) & 15)
        return sfg_fail(ctx, SFG_EINVAL, "XG and XP must be 16-byte aligned");
    return sfg_score_impl(ctx, LG, XG, XP, K, storage, edge_ids, ne, mode, scores_out, nullptr,
                          nullptr);
}

sfg_status sfg_affinity(sfg_ctx* ctx, const sfg_graph* L, const float* X, int K,
                        double* delta_out) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!L) return sfg_fail(ctx, SFG_EINVAL, "graph is NULL");
    if (K < 1) return sfg_fail(ctx, SFG_EINVAL, "K must be >= 1");
    SFG_TRY(sfg_check_dev(ctx, X, "X"));
    if (L->m > 0) SFG_TRY(sfg_check_dev(ctx, delta_out, "delta_out"));
    return sfg_affinity_impl(ctx, L, X, K, SFG_F32, delta_out);
}

}  // extern "C"
