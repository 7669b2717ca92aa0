// Maximum-weight spanning forest (the spanning-tree backbone of Sec. 3.1 / 3.4, where the paper
// approximates a low-stretch tree by a maximum spanning tree).
//
// Boruvka rounds under the strict order (weight descending, edge id ascending): every edge key is
// (FP32 weight bits << 32) | ~id, unique and ordered like that order, so the forest is unique and
// equal to Kruskal's. A round: (1) each component takes the largest key among edges leaving it
// (per row over its CSR entries, then one 64-bit atomicMax per row or per segment of a long
// row), (2) marks that edge and hooks to the component across it, (3) the 2-cycles
// that mutual choices create are broken toward the smaller label, (4) pointer jumping flattens the
// hook forest, (5) nodes are relabelled. Rounds repeat until no component has an outgoing edge.
#include "sfg_internal.cuh"

namespace {

constexpr int kBlock = 256;

__global__ void k_mst_init(int32_t n, int32_t* __restrict__ comp) {
    for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kBlock)
        comp[p] = (int32_t)p;
}

__global__ void k_mst_reset(int32_t n, unsigned long long* __restrict__ best, int* __restrict__ flag) {
    for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kBlock)
        best[p] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) *flag = 0;
}

// Each component's largest key among the edges leaving it, from the CSR rows: a group of 8 lanes
// takes kMstItems rows at a time, its lanes stride over each row's entries (the first entry of all
// rows is loaded before any later one), the group folds the largest key that leaves the row's
// component and issues one atomicMax for that component. Every
// edge leaving a component sits in the row of its endpoint inside it. SEG = false: rows
// [0, n), skipping rows longer than SFG_HEAVY_ROW; SEG = true: the fixed segments of those rows.
constexpr int kMstLanes = 8, kMstItems = 4;

struct MstItem {
    int32_t a, b, cp;
    unsigned long long best;
};

// Candidate key of CSR entry j of a row in component cp (0 if the entry stays inside it or the
// edge is not allowed).
__device__ __forceinline__ unsigned long long mst_key(int32_t j, int32_t cp, const int2* __restrict__ colval,
                                                      const int32_t* __restrict__ eid,
                                                      const uint8_t* __restrict__ allow,
                                                      const int32_t* __restrict__ comp,
                                                      const int32_t* __restrict__ key_id) {
    const int2 cv = colval[j];
    if (comp[cv.x] == cp) return 0ull;
    const int32_t e = eid[j];
    if (allow && !allow[e]) return 0ull;
    const uint32_t id = key_id ? (uint32_t)key_id[e] : (uint32_t)e;
    return ((unsigned long long)(uint32_t)cv.y << 32) | (unsigned long long)(~id);
}

template <bool SEG>
__global__ void __launch_bounds__(kBlock) k_mst_rows(int64_t nitems, const int32_t* __restrict__ row_ptr,
                                                     const int4* __restrict__ seg,
                                                     const int2* __restrict__ colval,
                                                     const int32_t* __restrict__ eid,
                                                     const uint8_t* __restrict__ allow,
                                                     const int32_t* __restrict__ comp,
                                                     const int32_t* __restrict__ key_id,
                                                     unsigned long long* __restrict__ best) {
    const int sub = threadIdx.x % kMstLanes;
    const int64_t g0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / kMstLanes;
    const int64_t ng = (int64_t)gridDim.x * kBlock / kMstLanes;
    const int64_t lg = g0 % (32 / kMstLanes);
    // kMstItems rows per group and iteration, so that as many independent load chains are in
    // flight; the same trip count for the whole warp, so the group folds below run converged
    for (int64_t i0 = g0 - lg; i0 < nitems; i0 += ng * kMstItems) {
        MstItem it[kMstItems];
        int32_t p[kMstItems];
#pragma unroll
        for (int u = 0; u < kMstItems; ++u) {
            const int64_t k = i0 + lg + (int64_t)u * ng;
            it[u].a = it[u].b = 0;
            p[u] = 0;
            if (k < nitems) {
                if (SEG) {
                    const int4 sg = seg[k];
                    p[u] = sg.x, it[u].a = sg.y, it[u].b = sg.z;
                } else {
                    p[u] = (int32_t)k, it[u].a = row_ptr[k], it[u].b = row_ptr[k + 1];
                    if (it[u].b - it[u].a > SFG_HEAVY_ROW) it[u].b = it[u].a;  // swept by segments
                }
            }
        }
        // the row's own label and its first entry (most rows of meshes and k-NN graphs have no
        // second) with the entry's edge id, all issued before any of them is used: the chain is
        // row bounds -> entry -> neighbour's label
        int2 cv[kMstItems];
        int32_t e[kMstItems];
#pragma unroll
        for (int u = 0; u < kMstItems; ++u) {
            it[u].cp = comp[p[u]];
            const int32_t j = it[u].a + sub;
            cv[u] = j < it[u].b ? colval[j] : make_int2(p[u], 0);
            e[u] = j < it[u].b ? eid[j] : 0;
        }
#pragma unroll
        for (int u = 0; u < kMstItems; ++u) {
            const bool out = comp[cv[u].x] != it[u].cp && (!allow || allow[e[u]]);
            const uint32_t id = key_id ? (uint32_t)key_id[e[u]] : (uint32_t)e[u];
            it[u].best = out ? ((unsigned long long)(uint32_t)cv[u].y << 32) |
                                   (unsigned long long)(~id)
                             : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kMstItems; ++u)
            for (int32_t j = it[u].a + sub + kMstLanes; j < it[u].b; j += kMstLanes) {
                const unsigned long long key = mst_key(j, it[u].cp, colval, eid, allow, comp, key_id);
                it[u].best = key > it[u].best ? key : it[u].best;
            }
#pragma unroll
        for (int u = 0; u < kMstItems; ++u) {
            unsigned long long local = it[u].best;
#pragma unroll
            for (int o = 1; o < kMstLanes; o <<= 1) {
                const unsigned long long q = __shfl_xor_sync(0xffffffffu, local, o);
                local = q > local ? q : local;
            }
            if (sub == 0 && local) atomicMax(&best[it[u].cp], local);
        }
    }
}

__global__ void k_mst_hook(int32_t n, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                           const int32_t* __restrict__ comp, const unsigned long long* __restrict__ best,
                           const int32_t* __restrict__ key_inv, int32_t* __restrict__ parent,
                           uint8_t* __restrict__ mask, int* __restrict__ flag) {
    for (int64_t r = (int64_t)blockIdx.x * kBlock + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * kBlock) {
        if (comp[r] != r) continue;  // only component labels act
        const unsigned long long b = best[r];
        if (b == 0ull) {
            parent[r] = (int32_t)r;
            continue;
        }
        const uint32_t id = ~(uint32_t)(b & 0xffffffffull);
        const uint32_t e = key_inv ? (uint32_t)key_inv[id] : id;
        mask[e] = 1;
        const int32_t a = comp[eu[e]], c = comp[ev[e]];
        parent[r] = (a == r) ? c : a;
        *flag = 1;
    }
}

__global__ void k_mst_break(int32_t n, const int32_t* __restrict__ comp, int32_t* __restrict__ parent) {
    for (int64_t r = (int64_t)blockIdx.x * kBlock + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * kBlock) {
        if (comp[r] != r) continue;
        const int32_t p = parent[r];
        // only the smaller label of a mutual pair writes, and it writes only its own entry
        if (p != r && p > r && parent[p] == (int32_t)r) parent[r] = (int32_t)r;
    }
}

// Pointer jumping in place on a forest (roots point to themselves): every node climbs up to
// kHops parents and stores the ancestor it reached; flag set while some node does not point at
// a root yet. Other threads' stores are read as they land: every stored value is an ancestor of
// its node, so any mix of old and new values is a valid forest with the same roots, and a node
// whose ancestors were already shortened climbs further (the reach grows geometrically from one
// launch to the next). Only component labels take part when comp != NULL.
constexpr int kHops = 8;

__global__ void k_jump_inplace(int32_t n, const int32_t* __restrict__ comp, int32_t* parent,
                               int* __restrict__ flag) {
    volatile int32_t* par = parent;
    for (int64_t r = (int64_t)blockIdx.x * kBlock + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * kBlock) {
        if (comp && comp[r] != r) continue;
        int32_t p = par[r];
#pragma unroll 1
        for (int h = 0; h < kHops; ++h) {
            const int32_t pp = par[p];
            if (pp == p) break;
            p = pp;
        }
        par[r] = p;
        if (par[p] != p) *flag = 1;
    }
}

__global__ void k_mst_relabel(int32_t n, int32_t* __restrict__ comp, const int32_t* __restrict__ parent) {
    for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kBlock)
        comp[p] = parent[comp[p]];
}

__global__ void k_count_u8(int64_t m, const uint8_t* __restrict__ mask,
                           unsigned long long* __restrict__ cnt) {
    unsigned long long c = 0;
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock)
        c += mask[e] != 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

}  // namespace

// Flatten a forest given by parent pointers (roots point to themselves) so that every entry
// points at its root: in-place jumping launches until no node moves (one launch when no path is
// longer than kHops; the reach multiplies by about kHops per launch otherwise).
sfg_status sfg_pointer_jump(sfg_ctx* ctx, int32_t n, const int32_t* comp, int32_t* parent) {
    if (n <= 0) return SFG_OK;
    Scratch s(ctx);
    int* flag;
    SFG_TRY(s.get(&flag, 1));
    int* h = nullptr;
    SFG_TRY(sfg_host_word(ctx, 1, &h));
    const int grid = sfg_grid(ctx, (const void*)k_jump_inplace, kBlock, 0, n);
    for (int it = 0; it < 64; ++it) {
        SFG_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
        sfg_tic(ctx, "jump");
        k_jump_inplace<<<grid, kBlock, 0, ctx->stream>>>(n, comp, parent, flag); ++ctx->launches;
        sfg_toc(ctx);
        SFG_LAUNCH_CHECK(ctx, "k_jump_inplace");
        SFG_CUDA(ctx, cudaMemcpyAsync(h, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (!*h) return SFG_OK;
    }
    return sfg_fail(ctx, SFG_ETIMEOUT, "pointer jumping did not converge");
}

sfg_status sfg_count_mask(sfg_ctx* ctx, const uint8_t* mask, int64_t m, int64_t* count_host) {
    Scratch s(ctx);
    unsigned long long* cnt;
    SFG_TRY(s.get(&cnt, 1));
    SFG_CUDA(ctx, cudaMemsetAsync(cnt, 0, 8, ctx->stream));
    if (m > 0) {
        k_count_u8<<<sfg_grid(ctx, (const void*)k_count_u8, kBlock, 0, m), kBlock, 0, ctx->stream>>>(
            m, mask, cnt); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_count_u8");
    }
    return sfg_read_i64(ctx, (const int64_t*)cnt, count_host);
}

sfg_status sfg_mst_impl(sfg_ctx* ctx, const sfg_graph* g, const uint8_t* allow, uint8_t* mask,
                        int64_t* n_tree, int32_t* comp_out, const int32_t* key_id,
                        const int32_t* key_inv) {
    const int32_t n = g->n;
    const int64_t m = g->m;
    if (m > 0) SFG_CUDA(ctx, cudaMemsetAsync(mask, 0, m, ctx->stream));
    if (m == 0) {
        if (n_tree) *n_tree = 0;
        if (comp_out && n > 0) {
            k_mst_init<<<sfg_grid(ctx, (const void*)k_mst_init, kBlock, 0, n), kBlock, 0, ctx->stream>>>(
                n, comp_out);
            ++ctx->launches;
            SFG_LAUNCH_CHECK(ctx, "k_mst_init");
        }
        return SFG_OK;
    }
    Scratch s(ctx);
    int32_t *comp, *parent;
    unsigned long long* best;
    int* flag;
    SFG_TRY(s.get(&comp, n));
    SFG_TRY(s.get(&parent, n));
    SFG_TRY(s.get(&best, n));
    SFG_TRY(s.get(&flag, 1));
    int* hflag = nullptr;  // pinned, written by the stream, read after a synchronisation
    SFG_TRY(sfg_host_word(ctx, 0, &hflag));
    const int gn = sfg_grid(ctx, (const void*)k_mst_hook, kBlock, 0, n);
    SFG_TRY(sfg_heavy_prepare(ctx, g));
    const int gr = sfg_grid(ctx, (const void*)k_mst_rows<false>, kBlock, 0, (int64_t)n * kMstLanes);
    const int gs = g->hv_n > 0 ? sfg_grid(ctx, (const void*)k_mst_rows<true>, kBlock, 0,
                                          g->hv_nseg * kMstLanes)
                               : 0;
    k_mst_init<<<gn, kBlock, 0, ctx->stream>>>(n, comp); ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_mst_init");
    // each round at least halves the number of components that still have outgoing edges
    for (int round = 0; round < 64; ++round) {
        sfg_tic(ctx, "mst_reset");
        k_mst_reset<<<gn, kBlock, 0, ctx->stream>>>(n, best, flag); ++ctx->launches;
        sfg_toc(ctx);
        sfg_tic(ctx, "mst_rows");
        k_mst_rows<false><<<gr, kBlock, 0, ctx->stream>>>(n, g->row_ptr, nullptr, g->colval, g->eid,
                                                          allow, comp, key_id, best);
        ++ctx->launches;
        if (gs > 0) {
            k_mst_rows<true><<<gs, kBlock, 0, ctx->stream>>>(g->hv_nseg, nullptr, g->hv_seg, g->colval,
                                                             g->eid, allow, comp, key_id, best);
            ++ctx->launches;
        }
        sfg_toc(ctx);
        sfg_tic(ctx, "mst_hook");
        k_mst_hook<<<gn, kBlock, 0, ctx->stream>>>(n, g->eu, g->ev, comp, best, key_inv, parent, mask,
                                                   flag);
        ++ctx->launches;
        sfg_toc(ctx);
        SFG_LAUNCH_CHECK(ctx, "k_mst_round");
        // The round's "any hook" flag travels with the pointer-jumping readback: a round in
        // which nothing hooks leaves every label its own parent, so break, jumping and relabel
        // change nothing and the check can wait for the next synchronisation.
        SFG_CUDA(ctx, cudaMemcpyAsync(hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        sfg_tic(ctx, "mst_break");
        k_mst_break<<<gn, kBlock, 0, ctx->stream>>>(n, comp, parent); ++ctx->launches;
        sfg_toc(ctx);
        SFG_TRY(sfg_pointer_jump(ctx, n, comp, parent));
        if (!*hflag) {
            if (n_tree) SFG_TRY(sfg_count_mask(ctx, mask, m, n_tree));
            if (comp_out)
                SFG_CUDA(ctx, cudaMemcpyAsync(comp_out, comp, sizeof(int32_t) * n,
                                              cudaMemcpyDeviceToDevice, ctx->stream));
            return SFG_OK;
        }
        sfg_tic(ctx, "mst_relabel");
        k_mst_relabel<<<gn, kBlock, 0, ctx->stream>>>(n, comp, parent); ++ctx->launches;
        sfg_toc(ctx);
        SFG_LAUNCH_CHECK(ctx, "k_mst_relabel");
    }
    return sfg_fail(ctx, SFG_ETIMEOUT, "spanning forest did not converge in 64 rounds");
}

extern "C" sfg_status sfg_spanning_tree(sfg_ctx* ctx, const sfg_graph* g, const uint8_t* allow,
                                        uint8_t* mask_out, int64_t* n_tree_host) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!g) return sfg_fail(ctx, SFG_EINVAL, "graph is NULL");
    if (g->m > 0) {
        SFG_TRY(sfg_check_dev(ctx, mask_out, "mask_out"));
        if (allow) SFG_TRY(sfg_check_dev(ctx, allow, "allow"));
    }
    return sfg_mst_impl(ctx, g, allow, mask_out, n_tree_host);
}
