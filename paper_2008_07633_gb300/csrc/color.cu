// Distance-1 colouring for the multicolour Gauss-Seidel smoother (Sec. 3.2 relaxes L x = 0 with
// Gauss-Seidel; nodes of one colour are pairwise non-adjacent, so a colour class is updated in
// parallel and the classes in order reproduce a sequential Gauss-Seidel sweep in that order).
//
// Jones-Plassmann rounds: node priority splitmix64(0x636f6c6f72 xor v), ties by the larger id. A
// round selects every uncoloured node that outranks all its uncoloured neighbours (one kernel),
// then gives each selected node the smallest colour no coloured neighbour holds (a second
// kernel, so no selection ever sees a colour written in the same round). Selected nodes are
// never adjacent, so the colouring is deterministic and proper.
#include "sfg_internal.cuh"

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ bool outranks(int32_t a, int32_t b) {
    const uint64_t pa = sfg_splitmix64(0x636f6c6f72ull ^ (uint64_t)(uint32_t)a);
    const uint64_t pb = sfg_splitmix64(0x636f6c6f72ull ^ (uint64_t)(uint32_t)b);
    return pa > pb || (pa == pb && a > b);
}

__global__ void k_jp_select(int32_t n, const int32_t* __restrict__ row_ptr,
                            const int2* __restrict__ colval, const int32_t* __restrict__ color,
                            uint8_t* __restrict__ sel, uint8_t* __restrict__ left) {
    for (int64_t v = blockIdx.x * (int64_t)kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock) {
        uint8_t top = 0;
        if (color[v] < 0) {
            top = 1;
            for (int32_t j = row_ptr[v]; j < row_ptr[v + 1] && top; ++j) {
                const int32_t u = colval[j].x;
                if (color[u] < 0 && outranks(u, (int32_t)v)) top = 0;
            }
        }
        sel[v] = top;
        left[v] = color[v] < 0 && !top;
    }
}

__global__ void k_jp_assign(int32_t n, const int32_t* __restrict__ row_ptr,
                            const int2* __restrict__ colval, const uint8_t* __restrict__ sel,
                            int32_t* __restrict__ color, int* __restrict__ maxc) {
    for (int64_t v = blockIdx.x * (int64_t)kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock) {
        if (!sel[v]) continue;
        // smallest colour absent among the coloured neighbours, 64 candidates at a time
        for (int32_t base = 0;; base += 64) {
            unsigned long long used = 0ull;
            for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
                const int32_t c = color[colval[j].x];
                if (c >= base && c < base + 64) used |= 1ull << (c - base);
            }
            if (used != ~0ull) {
                const int32_t c = base + __ffsll((long long)~used) - 1;
                color[v] = c;
                atomicMax(maxc, c);
                break;
            }
        }
    }
}

__global__ void k_iota_neg(int32_t n, int32_t* __restrict__ color) {
    for (int64_t v = blockIdx.x * (int64_t)kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock)
        color[v] = -1;
}

__global__ void k_color_keys(int32_t n, const int32_t* __restrict__ color,
                             uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
    for (int64_t v = blockIdx.x * (int64_t)kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock) {
        key[v] = ((uint64_t)(uint32_t)color[v] << 32) | (uint32_t)v;
        val[v] = (uint32_t)v;
    }
}

// order[i] = node of sorted position i; off[c] = first position of colour c (off[ncolors] = n).
__global__ void k_color_bounds(int32_t n, int32_t ncolors, const uint64_t* __restrict__ key,
                               const uint32_t* __restrict__ val, int32_t* __restrict__ order,
                               int64_t* __restrict__ off) {
    for (int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kBlock) {
        order[i] = (int32_t)val[i];
        const int32_t c = (int32_t)(key[i] >> 32);
        const int32_t cp = i == 0 ? -1 : (int32_t)(key[i - 1] >> 32);
        for (int32_t q = cp + 1; q <= c; ++q) off[q] = i;
        if (i == n - 1)
            for (int32_t q = c + 1; q <= ncolors; ++q) off[q] = n;
    }
}

}  // namespace

// Weights of the quantity a Gauss-Seidel / SOR sweep in (colour, id) order conserves: with
// M = (D - omega A_L)^-1 ((1 - omega) D + omega A_U), y^T M = y^T for y = (D - omega A_L)^T 1, i.e.
// y_p = d_p - omega * (weight of the edges from p to nodes later in the order). sum_p y_p =
// (2 - omega) * total weight > 0 for omega < 2. Constants are the fixed points, and the iteration
// converges to the constant (y . x0) / (y . 1); removing that y-weighted mean first keeps the
// block free of a constant the final projection would otherwise cancel in FP32.
// One thread per row (rows of meshes and k-NN graphs are short, and eight-lane groups measured
// slower there); rows longer than SFG_HEAVY_ROW are left to k_gs_weights_heavy.
__global__ void k_gs_weights(int32_t n, const int32_t* __restrict__ row_ptr,
                             const int2* __restrict__ colval, const int32_t* __restrict__ color,
                             double omega, double* __restrict__ y) {
    for (int64_t p = blockIdx.x * (int64_t)256 + threadIdx.x; p < n; p += (int64_t)gridDim.x * 256) {
        const int32_t a = row_ptr[p], b = row_ptr[p + 1];
        if (b - a > SFG_HEAVY_ROW) continue;
        const int32_t cp = color[p];
        double d = 0.0, later = 0.0;
        for (int32_t j = a; j < b; ++j) {
            const int32_t q = colval[j].x;
            const double w = (double)__int_as_float(colval[j].y);
            d += w;
            if (color[q] > cp || (color[q] == cp && q > (int32_t)p)) later += w;
        }
        y[p] = d - omega * later;
    }
}

// The same weights for the rows over SFG_HEAVY_ROW entries: one CTA of 256 threads per row, a
// fixed-order tree over the threads' partial sums.
__global__ void __launch_bounds__(256) k_gs_weights_heavy(int32_t nh, const int32_t* __restrict__ hrow,
                                                          const int32_t* __restrict__ row_ptr,
                                                          const int2* __restrict__ colval,
                                                          const int32_t* __restrict__ color,
                                                          double omega, double* __restrict__ y) {
    __shared__ double sd[256], sl[256];
    for (int32_t h = blockIdx.x; h < nh; h += gridDim.x) {
        const int32_t p = hrow[h], cp = color[p];
        double d = 0.0, later = 0.0;
        for (int32_t j = row_ptr[p] + threadIdx.x; j < row_ptr[p + 1]; j += 256) {
            const int2 cv = colval[j];
            const double w = (double)__int_as_float(cv.y);
            const int32_t cq = color[cv.x];
            d += w;
            if (cq > cp || (cq == cp && cv.x > p)) later += w;
        }
        sd[threadIdx.x] = d;
        sl[threadIdx.x] = later;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) {
                sd[threadIdx.x] += sd[threadIdx.x + o];
                sl[threadIdx.x] += sl[threadIdx.x + o];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) y[p] = sd[0] - omega * sl[0];
        __syncthreads();
    }
}

namespace {

template <typename K>
int grid_of(sfg_ctx* ctx, K kernel, int64_t work) {
    return sfg_grid(ctx, (const void*)kernel, kBlock, 0, work);
}

}  // namespace

sfg_status sfg_gs_prepare(sfg_ctx* ctx, const sfg_graph* Lc) {
    sfg_graph* L = const_cast<sfg_graph*>(Lc);  // the colouring is a cache of the graph
    if (L->gs_order) return SFG_OK;
    const int32_t n = L->n;
    cudaStream_t st = ctx->stream;
    int32_t *color = nullptr, *order = nullptr;
    SFG_TRY(sfg_alloc(ctx, (void**)&color, sizeof(int32_t) * (n > 0 ? n : 1)));
    sfg_status s = sfg_alloc(ctx, (void**)&order, sizeof(int32_t) * (n > 0 ? n : 1));
    if (s != SFG_OK) {
        sfg_free(ctx, color);
        return s;
    }
    struct Owner {  // released unless handed to the graph
        sfg_ctx* ctx;
        int32_t **a, **b;
        bool keep = false;
        ~Owner() {
            if (!keep) {
                sfg_free(ctx, *a);
                sfg_free(ctx, *b);
            }
        }
    } own{ctx, &color, &order};
    std::vector<int64_t> off(1, 0);
    if (n > 0) {
        Scratch t(ctx);
        uint8_t *sel, *left;
        int* maxc;
        SFG_TRY(t.get(&sel, n));
        SFG_TRY(t.get(&left, n));
        SFG_TRY(t.get(&maxc, 1));
        const int g = grid_of(ctx, k_jp_select, n);
        k_iota_neg<<<g, kBlock, 0, st>>>(n, color);
        SFG_CUDA(ctx, cudaMemsetAsync(maxc, 0, sizeof(int), st));
        ++ctx->launches;
        // rounds in batches of 4 between completion checks (a round after the last is a no-op)
        for (int round = 0;; round += 4) {
            if (round > n) return sfg_fail(ctx, SFG_ETIMEOUT, "colouring did not finish");
            for (int r = 0; r < 4; ++r) {
                k_jp_select<<<g, kBlock, 0, st>>>(n, L->row_ptr, L->colval, color, sel, left);
                k_jp_assign<<<g, kBlock, 0, st>>>(n, L->row_ptr, L->colval, sel, color, maxc);
            }
            ctx->launches += 8;
            SFG_LAUNCH_CHECK(ctx, "colouring round");
            int64_t remaining = 0;
            SFG_TRY(sfg_count_mask(ctx, left, n, &remaining));
            if (remaining == 0) break;
        }
        int hmax = 0;
        SFG_CUDA(ctx, cudaMemcpyAsync(&hmax, maxc, sizeof(int), cudaMemcpyDeviceToHost, st));
        SFG_CUDA(ctx, cudaStreamSynchronize(st));
        const int32_t ncolors = hmax + 1;
        uint64_t *k1, *k2;
        uint32_t *v1, *v2;
        int64_t* doff;
        SFG_TRY(t.get(&k1, n));
        SFG_TRY(t.get(&k2, n));
        SFG_TRY(t.get(&v1, n));
        SFG_TRY(t.get(&v2, n));
        SFG_TRY(t.get(&doff, (size_t)ncolors + 1));
        k_color_keys<<<grid_of(ctx, k_color_keys, n), kBlock, 0, st>>>(n, color, k1, v1);
        ++ctx->launches;
        int bits = 32;
        while ((1ll << (bits - 32)) < ncolors) ++bits;
        SFG_TRY(sfg_radix_sort_pairs(ctx, &k1, &v1, &k2, &v2, n, (bits + 7) / 8 * 8));
        k_color_bounds<<<grid_of(ctx, k_color_bounds, n), kBlock, 0, st>>>(n, ncolors, k1, v1, order,
                                                                           doff);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_color_bounds");
        off.assign((size_t)ncolors + 1, 0);
        SFG_CUDA(ctx, cudaMemcpyAsync(off.data(), doff, sizeof(int64_t) * (ncolors + 1),
                                      cudaMemcpyDeviceToHost, st));
        SFG_CUDA(ctx, cudaStreamSynchronize(st));
    }
    own.keep = true;
    L->gs_color = color;
    L->gs_order = order;
    L->gs_off = off;
    return SFG_OK;
}

// P shares G's nodes and has a subset of its edges, so G's colouring is a proper colouring of P:
// copy it (and its class order) instead of colouring P again.
sfg_status sfg_gs_inherit(sfg_ctx* ctx, const sfg_graph* Pc, const sfg_graph* G) {
    sfg_graph* P = const_cast<sfg_graph*>(Pc);
    if (P->gs_order) return SFG_OK;
    SFG_TRY(sfg_gs_prepare(ctx, G));
    const int32_t n = P->n;
    int32_t *color = nullptr, *order = nullptr;
    SFG_TRY(sfg_alloc(ctx, (void**)&color, sizeof(int32_t) * (n > 0 ? n : 1)));
    sfg_status s = sfg_alloc(ctx, (void**)&order, sizeof(int32_t) * (n > 0 ? n : 1));
    if (s != SFG_OK) {
        sfg_free(ctx, color);
        return s;
    }
    if (n > 0) {
        cudaError_t e = cudaMemcpyAsync(color, G->gs_color, sizeof(int32_t) * n,
                                        cudaMemcpyDeviceToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(order, G->gs_order, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice,
                                ctx->stream);
        if (e != cudaSuccess) {
            sfg_free(ctx, color);
            sfg_free(ctx, order);
            return sfg_cuda_fail(ctx, e, "colouring copy");
        }
    }
    P->gs_color = color;
    P->gs_order = order;
    P->gs_off = G->gs_off;
    return SFG_OK;
}

extern "C" sfg_status sfg_coloring(sfg_ctx* ctx, const sfg_graph* L, int32_t* color_out,
                                   int32_t* ncolors_host) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!L) return sfg_fail(ctx, SFG_EINVAL, "graph is NULL");
    if (L->n > 0 && color_out) SFG_TRY(sfg_check_dev(ctx, color_out, "color_out"));
    SFG_TRY(sfg_gs_prepare(ctx, L));
    if (color_out && L->n > 0)
        SFG_CUDA(ctx, cudaMemcpyAsync(color_out, L->gs_color, sizeof(int32_t) * L->n,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    if (ncolors_host) *ncolors_host = (int32_t)L->gs_off.size() - 1;
    return SFG_OK;
}
