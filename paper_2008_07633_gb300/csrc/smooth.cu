// Local spectral embedding (Sec. 3.2): K seeded random vectors orthogonal to the all-one vector,
// low-pass filtered by weighted-Jacobi sweeps on L x = 0, then projected (mean removed, unit RMS).
//
// The sweep X <- X - omega D^-1 L X is evaluated in its adjacency form
//     X'_p = (1 - omega) X_p + c_p * sum_q A(p,q) X_q,   c_p = omega / D(p,p) (FP64, rounded once),
// which is one CSR SpMM over the row-major block. Schedule: a group of LPR = K / E lanes owns a
// row (E = 4 FP32 or 8 BF16 entries per 16-byte lane vector); the group loads up to LPR (column,
// weight) pairs with one coalesced 8-byte load per lane, broadcasts them by shuffle, and issues all
// neighbour-row gathers before accumulating, so each warp keeps 32 / LPR rows and up to 32
// 16-byte gathers in flight. Every byte of the block is read and written once per sweep; the
// neighbour gathers are served by L2 on meshes (the band of rows between p - D and p + D fits).
//
// The first sweep also removes the initial column means (A-form sweeps map a constant column to
// itself, so J(X - 1 mu^T) = J(X) - 1 mu^T), and the last sweep accumulates the column sums and
// sums of squares the projection needs, so neither costs an extra pass over the block.
#include "sfg_internal.cuh"
#include "vec.cuh"

namespace {

constexpr int kBlock = 256;

// Gaussian draw j of the counter-based generator (see sfg.h): splitmix64 uniforms formed exactly
// in FP64, Box-Muller evaluated in FP32 (logf, cospif).
__device__ __forceinline__ float gaussian_draw(uint64_t seed, uint64_t j) {
    const uint64_t a = sfg_splitmix64(seed ^ sfg_splitmix64(2 * j));
    const uint64_t b = sfg_splitmix64(seed ^ sfg_splitmix64(2 * j + 1));
    const float u1 = (float)((double)((a >> 11) + 1) * 0x1.0p-53);
    const float u2 = (float)((double)(b >> 11) * 0x1.0p-53);
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

template <int LPR>
__device__ __forceinline__ unsigned group_mask(int lane) {
    if (LPR == 32) return 0xffffffffu;
    return ((1u << LPR) - 1u) << ((lane / LPR) * LPR);
}

// Per-thread column partials -> per-block FP64 partials part[block][2][K] (sums, sums of squares).
// Lanes with equal `sub` hold the same columns; fold them with xor-shuffles, then across warps in
// a fixed order, so the result is deterministic.
template <int LPR, int E>
__device__ __forceinline__ void block_column_partials(float (&s1)[E], float (&s2)[E],
                                                      double* __restrict__ part) {
    constexpr int K = LPR * E;
    __shared__ double ws[kBlock / 32][2 * K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, sub = lane % LPR;
#pragma unroll
    for (int o = LPR; o < 32; o <<= 1)
#pragma unroll
        for (int e = 0; e < E; ++e) {
            s1[e] += __shfl_xor_sync(0xffffffffu, s1[e], o);
            s2[e] += __shfl_xor_sync(0xffffffffu, s2[e], o);
        }
    if (lane < LPR)
#pragma unroll
        for (int e = 0; e < E; ++e) {
            ws[warp][sub * E + e] = (double)s1[e];
            ws[warp][K + sub * E + e] = (double)s2[e];
        }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * K; t += kBlock) {
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) acc += ws[w][t];
        part[(size_t)blockIdx.x * 2 * K + t] = acc;
    }
}

template <typename T, int LPR>
__global__ void __launch_bounds__(kBlock) k_init(int32_t n, uint64_t seed, T* __restrict__ X,
                                                 double* __restrict__ part) {
    constexpr int E = Vec<T>::E, K = LPR * E;
    const int lane = threadIdx.x & 31, sub = lane % LPR;
    const int64_t g0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / LPR;
    const int64_t ng = (int64_t)gridDim.x * kBlock / LPR;
    float s1[E], s2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) s1[e] = s2[e] = 0.f;
    for (int64_t row = g0; row < n; row += ng) {
        float x[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint64_t j = (uint64_t)row * K + sub * E + e;
            x[e] = Vec<T>::round(gaussian_draw(seed, j));
            s1[e] += x[e];
            s2[e] = fmaf(x[e], x[e], s2[e]);
        }
        Vec<T>::store(X + row * K + sub * E, x);
    }
    block_column_partials<LPR, E>(s1, s2, part);
}

template <typename T, int LPR, bool SUB_MU, bool STATS>
__global__ void __launch_bounds__(kBlock)
    k_jacobi(int32_t n, const int32_t* __restrict__ row_ptr, const int2* __restrict__ colval,
             const float* __restrict__ coef, float a_self, const T* __restrict__ X,
             T* __restrict__ Y, const float* __restrict__ mu, double* __restrict__ part) {
    constexpr int E = Vec<T>::E, K = LPR * E;
    const int lane = threadIdx.x & 31, sub = lane % LPR;
    const unsigned gm = group_mask<LPR>(lane);
    const int64_t g0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / LPR;
    const int64_t ng = (int64_t)gridDim.x * kBlock / LPR;
    float m[E], s1[E], s2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        m[e] = SUB_MU ? mu[sub * E + e] : 0.f;
        s1[e] = s2[e] = 0.f;
    }
    for (int64_t row = g0; row < n; row += ng) {
        const int32_t a = row_ptr[row], b = row_ptr[row + 1];
        float acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;
        for (int32_t j0 = a; j0 < b; j0 += LPR) {
            const int32_t j = j0 + sub;
            const int2 cv = j < b ? colval[j] : make_int2(0, 0);
            const int cnt = min(LPR, b - j0);
            float xv[LPR][E];
            float wv[LPR];
#pragma unroll
            for (int t = 0; t < LPR; ++t) {
                if (t < cnt) {
                    const int c = __shfl_sync(gm, cv.x, t, LPR);
                    wv[t] = __int_as_float(__shfl_sync(gm, cv.y, t, LPR));
                    Vec<T>::load(X + (int64_t)c * K + sub * E, xv[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < LPR; ++t)
                if (t < cnt)
#pragma unroll
                    for (int e = 0; e < E; ++e) acc[e] = fmaf(wv[t], xv[t][e], acc[e]);
        }
        float xs[E], y[E];
        Vec<T>::load(X + row * K + sub * E, xs);
        if (b > a) {
            const float cp = coef[row];
#pragma unroll
            for (int e = 0; e < E; ++e) y[e] = fmaf(cp, acc[e], a_self * xs[e]);
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) y[e] = xs[e];
        }
#pragma unroll
        for (int e = 0; e < E; ++e) y[e] -= m[e];
        Vec<T>::store(Y + row * K + sub * E, y);
        if (STATS)
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const float r = Vec<T>::round(y[e]);
                s1[e] += r;
                s2[e] = fmaf(r, r, s2[e]);
            }
    }
    if (STATS) block_column_partials<LPR, E>(s1, s2, part);
}

// Fold the per-block partials in block order (FP64). proj = 0: mean only (mu = S1 / n).
// proj = 1: mean and scale = 1 / RMS of the centred column (1 if the column is zero).
__global__ void k_finalize(const double* __restrict__ part, int nblocks, int K, int32_t n,
                           int proj, float* __restrict__ mean, float* __restrict__ scale) {
    const int k = threadIdx.x;
    if (k >= K) return;
    double s1 = 0.0, s2 = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        s1 += part[(size_t)b * 2 * K + k];
        s2 += part[(size_t)b * 2 * K + K + k];
    }
    const double mu = s1 / (double)n;
    mean[k] = (float)mu;
    if (proj) {
        const double var = s2 / (double)n - mu * mu;
        const double rms = var > 0.0 ? sqrt(var) : 0.0;
        scale[k] = rms > 0.0 ? (float)(1.0 / rms) : 1.0f;
    }
}

template <typename T, int LPR>
__global__ void __launch_bounds__(kBlock) k_project(int32_t n, const T* __restrict__ X,
                                                    T* __restrict__ Y, const float* __restrict__ mean,
                                                    const float* __restrict__ scale) {
    constexpr int E = Vec<T>::E, K = LPR * E;
    const int64_t total = (int64_t)n * LPR;  // 16-byte vectors
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * kBlock) {
        const int c0 = (int)(i % LPR) * E;
        float x[E];
        Vec<T>::load(X + i * E, x);
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = (x[e] - mean[c0 + e]) * scale[c0 + e];
        Vec<T>::store(Y + i * E, x);
        (void)K;
    }
}

__global__ void k_coef(int32_t n, const double* __restrict__ deg, double omega,
                       float* __restrict__ coef) {
    for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kBlock)
        coef[p] = deg[p] > 0.0 ? (float)(omega / deg[p]) : 0.0f;
}

template <typename T, int LPR>
struct Smoother {
    using Elem = T;
    static constexpr int E = Vec<T>::E, K = LPR * E;

    static int grid_jacobi(sfg_ctx* ctx, int32_t n) {
        return sfg_grid(ctx, (const void*)k_jacobi<T, LPR, false, true>, kBlock, 0,
                        (int64_t)n * LPR);
    }

    static sfg_status sweep(sfg_ctx* ctx, const sfg_graph* L, const float* coef, float a_self,
                            const T* X, T* Y, const float* mu, double* part, bool sub_mu,
                            bool stats, int grid) {
        const int32_t n = L->n;
        sfg_tic(ctx, "jacobi");
        if (sub_mu && stats)
            k_jacobi<T, LPR, true, true><<<grid, kBlock, 0, ctx->stream>>>(
                n, L->row_ptr, L->colval, coef, a_self, X, Y, mu, part);
        else if (sub_mu)
            k_jacobi<T, LPR, true, false><<<grid, kBlock, 0, ctx->stream>>>(
                n, L->row_ptr, L->colval, coef, a_self, X, Y, mu, part);
        else if (stats)
            k_jacobi<T, LPR, false, true><<<grid, kBlock, 0, ctx->stream>>>(
                n, L->row_ptr, L->colval, coef, a_self, X, Y, mu, part);
        else
            k_jacobi<T, LPR, false, false><<<grid, kBlock, 0, ctx->stream>>>(
                n, L->row_ptr, L->colval, coef, a_self, X, Y, mu, part);
        sfg_toc(ctx);
        SFG_LAUNCH_CHECK(ctx, "k_jacobi");
        return SFG_OK;
    }

    static sfg_status smooth(sfg_ctx* ctx, const sfg_graph* L, int steps, double omega,
                             uint64_t seed, T* X_out) {
        const int32_t n = L->n;
        const int grid = grid_jacobi(ctx, n);
        Scratch s(ctx);
        T* buf;
        float *coef, *mu, *scale;
        double* part;
        SFG_TRY(s.get(&buf, (size_t)n * K));
        SFG_TRY(s.get(&coef, (size_t)n));
        SFG_TRY(s.get(&mu, K));
        SFG_TRY(s.get(&scale, K));
        SFG_TRY(s.get(&part, (size_t)grid * 2 * K));
        k_coef<<<sfg_grid(ctx, (const void*)k_coef, kBlock, 0, n), kBlock, 0, ctx->stream>>>(
            n, L->deg, omega, coef);
        SFG_LAUNCH_CHECK(ctx, "k_coef");
        // ping-pong so that the last sweep writes `buf` and the projection writes X_out
        T* cur = (steps % 2 == 0) ? buf : X_out;
        T* nxt = (cur == buf) ? X_out : buf;
        sfg_tic(ctx, "init");
        k_init<T, LPR><<<grid, kBlock, 0, ctx->stream>>>(n, seed, cur, part);
        sfg_toc(ctx);
        SFG_LAUNCH_CHECK(ctx, "k_init");
        k_finalize<<<1, 64, 0, ctx->stream>>>(part, grid, K, n, steps == 0 ? 1 : 0, mu, scale);
        SFG_LAUNCH_CHECK(ctx, "k_finalize");
        for (int t = 1; t <= steps; ++t) {
            SFG_TRY(sweep(ctx, L, coef, (float)(1.0 - omega), cur, nxt, mu, part, t == 1,
                          t == steps, grid));
            std::swap(cur, nxt);
        }
        if (steps > 0) {
            k_finalize<<<1, 64, 0, ctx->stream>>>(part, grid, K, n, 1, mu, scale);
            SFG_LAUNCH_CHECK(ctx, "k_finalize");
        }
        sfg_tic(ctx, "project");
        k_project<T, LPR><<<sfg_grid(ctx, (const void*)k_project<T, LPR>, kBlock, 0,
                                     (int64_t)n * LPR),
                            kBlock, 0, ctx->stream>>>(n, cur, X_out, mu, scale);
        sfg_toc(ctx);
        SFG_LAUNCH_CHECK(ctx, "k_project");
        return SFG_OK;
    }

    static sfg_status jacobi(sfg_ctx* ctx, const sfg_graph* L, int steps, double omega, T* X) {
        const int32_t n = L->n;
        const int grid = grid_jacobi(ctx, n);
        Scratch s(ctx);
        T* buf;
        float* coef;
        SFG_TRY(s.get(&buf, (size_t)n * K));
        SFG_TRY(s.get(&coef, (size_t)n));
        k_coef<<<sfg_grid(ctx, (const void*)k_coef, kBlock, 0, n), kBlock, 0, ctx->stream>>>(
            n, L->deg, omega, coef);
        SFG_LAUNCH_CHECK(ctx, "k_coef");
        T* cur = X;
        T* nxt = buf;
        for (int t = 1; t <= steps; ++t) {
            SFG_TRY(sweep(ctx, L, coef, (float)(1.0 - omega), cur, nxt, nullptr, nullptr, false,
                          false, grid));
            std::swap(cur, nxt);
        }
        if (cur != X)
            SFG_CUDA(ctx, cudaMemcpyAsync(X, cur, sizeof(T) * (size_t)n * K,
                                          cudaMemcpyDeviceToDevice, ctx->stream));
        return SFG_OK;
    }
};

template <typename F>
sfg_status dispatch(int K, sfg_dtype dt, F&& f) {
    if (dt == SFG_F32) {
        switch (K) {
            case 4: return f(Smoother<float, 1>());
            case 8: return f(Smoother<float, 2>());
            case 16: return f(Smoother<float, 4>());
            case 32: return f(Smoother<float, 8>());
            case 64: return f(Smoother<float, 16>());
        }
    } else if (dt == SFG_BF16) {
        switch (K) {
            case 8: return f(Smoother<__nv_bfloat16, 1>());
            case 16: return f(Smoother<__nv_bfloat16, 2>());
            case 32: return f(Smoother<__nv_bfloat16, 4>());
            case 64: return f(Smoother<__nv_bfloat16, 8>());
        }
    }
    return SFG_EUNSUPPORTED;
}

}  // namespace

bool sfg_k_supported(int K, sfg_dtype dt) {
    if (dt == SFG_F32) return K == 4 || K == 8 || K == 16 || K == 32 || K == 64;
    if (dt == SFG_BF16) return K == 8 || K == 16 || K == 32 || K == 64;
    return false;
}

sfg_status sfg_smooth_impl(sfg_ctx* ctx, const sfg_graph* L, int K, int steps, double omega,
                           uint64_t seed, sfg_dtype storage, void* X_out) {
    return dispatch(K, storage, [&](auto S) {
        using Sm = decltype(S);
        return Sm::smooth(ctx, L, steps, omega, seed, static_cast<typename Sm::Elem*>(X_out));
    });
}

static sfg_status check_smooth_args(sfg_ctx* ctx, const sfg_graph* L, int K, int steps,
                                    double omega, sfg_dtype storage, const void* X) {
    if (!L) return sfg_fail(ctx, SFG_EINVAL, "graph is NULL");
    if (!sfg_k_supported(K, storage))
        return sfg_fail(ctx, SFG_EUNSUPPORTED, "K=%d unsupported for dtype %d", K, (int)storage);
    if (steps < 0) return sfg_fail(ctx, SFG_EINVAL, "steps must be >= 0");
    if (!(omega > 0.0 && omega <= 1.0)) return sfg_fail(ctx, SFG_EINVAL, "omega must be in (0, 1]");
    SFG_TRY(sfg_check_dev(ctx, X, "X"));
    if (((uintptr_t)X & 15) != 0) return sfg_fail(ctx, SFG_EINVAL, "X must be 16-byte aligned");
    return SFG_OK;
}

extern "C" {

sfg_status sfg_smooth(sfg_ctx* ctx, const sfg_graph* L, int K, int steps, double omega,
                      uint64_t seed, sfg_dtype storage, void* X_out) {
    if (!ctx) return SFG_EINVAL;
    SFG_TRY(check_smooth_args(ctx, L, K, steps, omega, storage, X_out));
    return sfg_smooth_impl(ctx, L, K, steps, omega, seed, storage, X_out);
}

sfg_status sfg_jacobi(sfg_ctx* ctx, const sfg_graph* L, int K, int steps, double omega,
                      sfg_dtype storage, void* X_inout) {
    if (!ctx) return SFG_EINVAL;
    SFG_TRY(check_smooth_args(ctx, L, K, steps, omega, storage, X_inout));
    return dispatch(K, storage, [&](auto S) {
        using Sm = decltype(S);
        return Sm::jacobi(ctx, L, steps, omega, static_cast<typename Sm::Elem*>(X_inout));
    });
}

}  // extern "C"
