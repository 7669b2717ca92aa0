// One level of spectral coarsening (Sec. 3.2) and the sparsifier backward mapping (Sec. 3.4,
// the backward-mapping step of Algorithm 1).
//
// Aggregation: every node hooks to the neighbour of smallest algebraic distance (ties: smaller
// id). Under that strict choice the hook graph has no cycle longer than two, so breaking each
// mutual pair toward its smaller node leaves a forest; pointer jumping labels its trees, and the
// trees are the aggregation sets, numbered by increasing smallest member. The Galerkin coarse
// Laplacian H^-T L H^+ is the canonical form of the relabelled edge list (agg[u], agg[v], w), so
// it reuses the canonicalisation of the Laplacian build.
#include "sfg_internal.cuh"

namespace {

constexpr int kBlock = 256;

__global__ void k_hook(int32_t n, const int32_t* __restrict__ row_ptr, const int2* __restrict__ colval,
                       const int32_t* __restrict__ eid, const double* __restrict__ delta,
                       int32_t* __restrict__ hook) {
    for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kBlock) {
        int32_t best = -1;
        double bd = 0.0;
        for (int32_t j = row_ptr[p]; j < row_ptr[p + 1]; ++j) {
            const double d = delta[eid[j]];
            const int32_t q = colval[j].x;
            if (best < 0 || d < bd || (d == bd && q < best)) {
                best = q;
                bd = d;
            }
        }
        hook[p] = best < 0 ? (int32_t)p : best;
    }
}

// parent = hook, except the smaller node of a mutual pair, which becomes a root.
__global__ void k_hook_forest(int32_t n, const int32_t* __restrict__ hook, int32_t* __restrict__ parent) {
    for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kBlock) {
        const int32_t h = hook[p];
        parent[p] = (h != p && hook[h] == p && p < h) ? (int32_t)p : h;
    }
}

__global__ void k_min_member(int32_t n, const int32_t* __restrict__ root, int32_t* __restrict__ minm) {
    for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kBlock)
        atomicMin(&minm[root[p]], (int32_t)p);
}

__global__ void k_is_first(int32_t n, const int32_t* __restrict__ root, const int32_t* __restrict__ minm,
                           uint8_t* __restrict__ first) {
    for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kBlock)
        first[p] = minm[root[p]] == p;
}

__global__ void k_agg_label(int32_t n, const int32_t* __restrict__ root, const int32_t* __restrict__ minm,
                            const int64_t* __restrict__ rank, int32_t* __restrict__ agg) {
    for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kBlock)
        agg[p] = (int32_t)rank[minm[root[p]]];
}

__global__ void k_relabel_edges(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                                const int32_t* __restrict__ agg, int32_t* __restrict__ cu,
                                int32_t* __restrict__ cv) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock) {
        cu[e] = agg[eu[e]];
        cv[e] = agg[ev[e]];
    }
}

__global__ void k_inner_allow(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                              const int32_t* __restrict__ agg, uint8_t* __restrict__ allow) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock)
        allow[e] = agg[eu[e]] == agg[ev[e]];
}

__global__ void k_inter_best(int64_t m, const float* __restrict__ ew, const int32_t* __restrict__ f2c,
                             const uint8_t* __restrict__ pmask_c, unsigned long long* __restrict__ best) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock) {
        const int32_t c = f2c[e];
        if (c < 0 || !pmask_c[c]) continue;
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(ew[e]) << 32) | (unsigned long long)(~(uint32_t)e);
        atomicMax(&best[c], key);
    }
}

__global__ void k_inter_mark(int64_t mc, const unsigned long long* __restrict__ best,
                             uint8_t* __restrict__ pmask_f) {
    for (int64_t c = (int64_t)blockIdx.x * kBlock + threadIdx.x; c < mc;
         c += (int64_t)gridDim.x * kBlock) {
        const unsigned long long b = best[c];
        if (b) pmask_f[~(uint32_t)(b & 0xffffffffull)] = 1;
    }
}

template <typename K>
int grid_of(sfg_ctx* ctx, K kernel, int64_t work) {
    return sfg_grid(ctx, (const void*)kernel, kBlock, 0, work);
}

}  // namespace

// Aggregation sets from per-edge distances delta (FP64). Writes agg[n], returns the set count.
static sfg_status aggregate(sfg_ctx* ctx, const sfg_graph* L, const double* delta, int32_t* agg,
                            int32_t* nc_host) {
    const int32_t n = L->n;
    Scratch s(ctx);
    int32_t *hook, *root, *minm;
    uint8_t* first;
    int64_t* rank;
    SFG_TRY(s.get(&hook, n));
    SFG_TRY(s.get(&root, n));
    SFG_TRY(s.get(&minm, n));
    SFG_TRY(s.get(&first, n));
    SFG_TRY(s.get(&rank, (size_t)n + 1));
    const int gn = grid_of(ctx, k_hook, n);
    k_hook<<<gn, kBlock, 0, ctx->stream>>>(n, L->row_ptr, L->colval, L->eid, delta, hook); ++ctx->launches;
    k_hook_forest<<<gn, kBlock, 0, ctx->stream>>>(n, hook, root); ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_hook");
    SFG_TRY(sfg_pointer_jump(ctx, n, nullptr, root));
    SFG_CUDA(ctx, cudaMemsetAsync(minm, 0x7f, sizeof(int32_t) * n, ctx->stream));
    k_min_member<<<gn, kBlock, 0, ctx->stream>>>(n, root, minm); ++ctx->launches;
    k_is_first<<<gn, kBlock, 0, ctx->stream>>>(n, root, minm, first); ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_min_member");
    SFG_TRY(sfg_scan_u8(ctx, first, rank, n));
    k_agg_label<<<gn, kBlock, 0, ctx->stream>>>(n, root, minm, rank, agg); ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_agg_label");
    int64_t nc = 0;
    SFG_TRY(sfg_read_i64(ctx, rank + n, &nc));
    *nc_host = (int32_t)nc;
    return SFG_OK;
}

sfg_status sfg_coarsen_impl(sfg_ctx* ctx, const sfg_graph* L, const void* X, int K,
                            sfg_dtype storage, int32_t* agg, int32_t* f2c, int32_t* nc_host,
                            sfg_graph** coarse) {
    *coarse = nullptr;
    Scratch s(ctx);
    double* delta;
    int32_t *cu, *cv;
    SFG_TRY(s.get(&delta, L->m));
    SFG_TRY(s.get(&cu, L->m));
    SFG_TRY(s.get(&cv, L->m));
    SFG_TRY(sfg_affinity_impl(ctx, L, X, K, storage, delta));
    int32_t nc = 0;
    SFG_TRY(aggregate(ctx, L, delta, agg, &nc));
    if (L->m > 0) {
        k_relabel_edges<<<grid_of(ctx, k_relabel_edges, L->m), kBlock, 0, ctx->stream>>>(
            L->m, L->eu, L->ev, agg, cu, cv); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_relabel_edges");
    }
    SFG_TRY(sfg_build_graph(ctx, nc, L->m, cu, cv, L->ew, false, coarse, f2c));
    *nc_host = nc;
    return SFG_OK;
}

sfg_status sfg_backward_impl(sfg_ctx* ctx, const sfg_graph* fine, const int32_t* agg,
                             const int32_t* f2c, const sfg_graph* coarse, const uint8_t* pmask_c,
                             uint8_t* pmask_f) {
    Scratch s(ctx);
    uint8_t* allow;
    unsigned long long* best;
    SFG_TRY(s.get(&allow, fine->m));
    SFG_TRY(s.get(&best, coarse->m));
    if (fine->m > 0) {
        k_inner_allow<<<grid_of(ctx, k_inner_allow, fine->m), kBlock, 0, ctx->stream>>>(
            fine->m, fine->eu, fine->ev, agg, allow); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_inner_allow");
    }
    SFG_TRY(sfg_mst_impl(ctx, fine, allow, pmask_f, nullptr));  // inner-cluster trees
    if (coarse->m > 0 && fine->m > 0) {
        SFG_CUDA(ctx, cudaMemsetAsync(best, 0, 8 * coarse->m, ctx->stream));
        k_inter_best<<<grid_of(ctx, k_inter_best, fine->m), kBlock, 0, ctx->stream>>>(
            fine->m, fine->ew, f2c, pmask_c, best); ++ctx->launches;
        k_inter_mark<<<grid_of(ctx, k_inter_mark, coarse->m), kBlock, 0, ctx->stream>>>(
            coarse->m, best, pmask_f); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_inter");
    }
    return SFG_OK;
}

extern "C" {

sfg_status sfg_coarsen(sfg_ctx* ctx, const sfg_graph* L, const void* X, int K, sfg_dtype storage,
                       int32_t* agg_out, int32_t* fine2coarse_out, int32_t* n_coarse_host,
                       sfg_graph** coarse_out) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!L || !coarse_out || !n_coarse_host) return sfg_fail(ctx, SFG_EINVAL, "NULL argument");
    if (K < 1) return sfg_fail(ctx, SFG_EINVAL, "K must be >= 1");
    if (storage != SFG_F32 && storage != SFG_BF16)
        return sfg_fail(ctx, SFG_EINVAL, "unknown storage type %d", (int)storage);
    SFG_TRY(sfg_check_dev(ctx, X, "X"));
    SFG_TRY(sfg_check_dev(ctx, agg_out, "agg_out"));
    if (fine2coarse_out && L->m > 0) SFG_TRY(sfg_check_dev(ctx, fine2coarse_out, "fine2coarse_out"));
    Scratch s(ctx);
    int32_t* f2c = fine2coarse_out;
    if (!f2c) SFG_TRY(s.get(&f2c, L->m));
    return sfg_coarsen_impl(ctx, L, X, K, storage, agg_out, f2c, n_coarse_host, coarse_out);
}

sfg_status sfg_backward_map(sfg_ctx* ctx, const sfg_graph* fine, const int32_t* agg,
                            const int32_t* fine2coarse, const sfg_graph* coarse,
                            const uint8_t* pmask_c, uint8_t* pmask_f) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!fine || !coarse) return sfg_fail(ctx, SFG_EINVAL, "graph is NULL");
    SFG_TRY(sfg_check_dev(ctx, agg, "agg"));
    if (fine->m > 0) {
        SFG_TRY(sfg_check_dev(ctx, fine2coarse, "fine2coarse"));
        SFG_TRY(sfg_check_dev(ctx, pmask_f, "pmask_f"));
    }
    if (coarse->m > 0) SFG_TRY(sfg_check_dev(ctx, pmask_c, "pmask_c"));
    return sfg_backward_impl(ctx, fine, agg, fine2coarse, coarse, pmask_c, pmask_f);
}

}  // extern "C"
