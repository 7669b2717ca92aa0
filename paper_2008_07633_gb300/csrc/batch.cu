// Batched flat sparsification of many graphs (a batch of independent problems, e.g. many small
// k-NN graphs) in one set of launches.
//
// The work splits in two. A batch plan (sfg_batch_create) holds everything that depends on the
// graphs only: their disjoint union, the spanning forests, the union of the forests' Laplacians,
// the candidate edges and per-graph budgets, the heavy-row segments and the sweep's tuned tile
// shape. Running the plan (sfg_batch_run) does the numeric part -- seeded blocks, sweeps on both
// unions, per-graph projection statistics, scores, per-graph top-k, masks -- as kernel launches and
// stream-ordered allocations only: no host synchronisation, so a run can be captured in a CUDA
// graph and replayed.
//
// The graphs are joined into their disjoint union U: canonical lists, CSR rows and entries are
// concatenated with node and edge offsets, which keeps every list sorted and every edge id order,
// so no sort is needed. On U, one Boruvka run gives every graph's spanning forest (the forests of
// disjoint components are independent and the strict edge order is preserved), one launch per
// Jacobi sweep smooths every graph, and the per-graph parts -- the seeded blocks, their mean
// removal, the projection scales, the budgets and the top-k -- are segmented by graph. Each
// graph's result is the one sfg_sparsify gives for it alone with the same parameters (up to FP32
// summation order in the column statistics).
//
// Locality order (optional): the nodes of each graph are renumbered by breadth-first level from a
// pseudo-peripheral root (a stable sort by (graph, level), so ties keep their order), and the
// plan works on the relabelled union. Neighbours then sit a few levels apart instead of anywhere
// in the graph, so the sweeps' and the scorer's row gathers hit L2 (random-order k-NN graphs: about
// twice as fast). Everything that decides the result keeps the original numbering: the seeded row
// of a node is drawn from its original id, the spanning forest breaks weight ties by original edge
// id, and top-k selects by original edge id; the masks come out in the original edge order. The
// result is the unreordered plan's up to FP32 summation order in the sweeps and statistics.
#include <cmath>
#include <vector>

#include "sfg_internal.cuh"

namespace {

constexpr int kBlock = 256;

struct GDesc {
    const int32_t *eu, *ev;
    const float* ew;
    const int32_t* row_ptr;
    const int2* colval;
    const int32_t* eid;
    const double *deg, *invdeg;
    int32_t node_off;
    int64_t edge_off;
};

template <typename O>
__device__ __forceinline__ int seg_of(const O* __restrict__ off, int ng, int64_t i) {
    int lo = 0, hi = ng;  // last g with off[g] <= i
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if ((int64_t)off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_union_edges(int64_t m, const GDesc* __restrict__ d, int ng,
                              const int64_t* __restrict__ eoff, int32_t* __restrict__ eu,
                              int32_t* __restrict__ ev, float* __restrict__ ew) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock) {
        const int g = seg_of(eoff, ng, e);
        const int64_t l = e - eoff[g];
        eu[e] = d[g].eu[l] + d[g].node_off;
        ev[e] = d[g].ev[l] + d[g].node_off;
        ew[e] = d[g].ew[l];
    }
}

__global__ void k_union_rows(int32_t n, int64_t m, const GDesc* __restrict__ d, int ng,
                             const int32_t* __restrict__ noff, int32_t* __restrict__ row_ptr,
                             double* __restrict__ deg, double* __restrict__ invdeg) {
    for (int64_t r = (int64_t)blockIdx.x * kBlock + threadIdx.x; r <= n;
         r += (int64_t)gridDim.x * kBlock) {
        if (r == n) {
            row_ptr[n] = (int32_t)(2 * m);
            continue;
        }
        const int g = seg_of(noff, ng, r);
        const int64_t l = r - noff[g];
        row_ptr[r] = d[g].row_ptr[l] + (int32_t)(2 * d[g].edge_off);
        deg[r] = d[g].deg[l];
        invdeg[r] = d[g].invdeg[l];
    }
}

__global__ void k_union_entries(int64_t m, const GDesc* __restrict__ d, int ng,
                                const int64_t* __restrict__ eoff, int2* __restrict__ colval,
                                int32_t* __restrict__ eid) {
    for (int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x; j < 2 * m;
         j += (int64_t)gridDim.x * kBlock) {
        const int g = seg_of(eoff, ng, j >> 1);  // graph g owns entries [2 eoff[g], 2 eoff[g+1])
        const int64_t l = j - 2 * eoff[g];
        const int2 cv = d[g].colval[l];
        colval[j] = make_int2(cv.x + d[g].node_off, cv.y);
        eid[j] = d[g].eid[l] + (int32_t)d[g].edge_off;
    }
}

// per-graph count of set mask entries (edge ranges eoff)
__global__ void k_seg_count(int64_t m, const uint8_t* __restrict__ mask, int ng,
                            const int64_t* __restrict__ eoff, unsigned long long* __restrict__ cnt) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock) {
        const bool on = mask[e] != 0;
        const unsigned bin = on ? (unsigned)seg_of(eoff, ng, e) : 0xffffffffu;
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, bin);
        if (on && (__ffs(peers) - 1) == (int)(threadIdx.x & 31))
            atomicAdd(&cnt[bin], (unsigned long long)__popc(peers));
    }
}

__global__ void k_not(int64_t m, const uint8_t* __restrict__ mask, uint8_t* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock)
        out[e] = mask[e] == 0;
}

__global__ void k_compact(int64_t m, const uint8_t* __restrict__ flag, const int64_t* __restrict__ pos,
                          int32_t* __restrict__ ids) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock)
        if (flag[e]) ids[pos[e]] = (int32_t)e;
}

__global__ void k_mark(int64_t k, const int32_t* __restrict__ ids, uint8_t* __restrict__ mask) {
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < k;
         i += (int64_t)gridDim.x * kBlock)
        mask[ids[i]] = 1;
}

__global__ void k_split(int64_t m, const uint8_t* __restrict__ mask, int ng,
                        const int64_t* __restrict__ eoff, uint8_t* const* __restrict__ outs) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock) {
        const int g = seg_of(eoff, ng, e);
        outs[g][e - eoff[g]] = mask[e];
    }
}

// ---- locality order ---------------------------------------------------------------------------
__global__ void k_bfs_seed(int ng, const int32_t* __restrict__ noff, const int32_t* __restrict__ roots,
                           int32_t* __restrict__ level) {
    for (int g = (int)(blockIdx.x * kBlock + threadIdx.x); g < ng; g += gridDim.x * kBlock)
        if (noff[g + 1] > noff[g]) level[roots ? roots[g] : noff[g]] = 0;
}

// one breadth-first level: every node of level cur labels its unlabelled neighbours cur + 1 (all
// writers of a node store the same value)
__global__ void k_bfs_step(int32_t n, const int32_t* __restrict__ row_ptr, const int2* __restrict__ colval,
                           int32_t cur, int32_t* __restrict__ level, int* __restrict__ flag) {
    for (int64_t v = (int64_t)blockIdx.x * kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock) {
        if (level[v] != cur) continue;
        bool any = false;
        for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
            const int32_t w = colval[j].x;
            if (level[w] < 0) {
                level[w] = cur + 1;
                any = true;
            }
        }
        if (any) *flag = 1;
    }
}

// per graph, the labelled node of the largest level (ties: the smallest id)
__global__ void k_bfs_far(int32_t n, const int32_t* __restrict__ noff, int ng,
                          const int32_t* __restrict__ level, unsigned long long* __restrict__ best) {
    for (int64_t v = (int64_t)blockIdx.x * kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock) {
        const int32_t l = level[v];
        if (l < 0) continue;
        const int g = seg_of(noff, ng, v);
        atomicMax(&best[g], ((unsigned long long)(uint32_t)l << 32) | (unsigned long long)(~(uint32_t)v));
    }
}

__global__ void k_bfs_roots(int ng, const unsigned long long* __restrict__ best,
                            const int32_t* __restrict__ noff, int32_t* __restrict__ roots) {
    for (int g = (int)(blockIdx.x * kBlock + threadIdx.x); g < ng; g += gridDim.x * kBlock)
        roots[g] = best[g] ? (int32_t)(~(uint32_t)(best[g] & 0xffffffffull)) : noff[g];
}

// sort key (graph, level; unreached nodes after the deepest level) and the node id as value
__global__ void k_order_keys(int32_t n, const int32_t* __restrict__ noff, int ng,
                             const int32_t* __restrict__ level, int32_t unreached, int lbits,
                             uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    for (int64_t v = (int64_t)blockIdx.x * kBlock + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * kBlock) {
        const int32_t l = level[v] >= 0 ? level[v] : unreached;
        keys[v] = ((uint64_t)seg_of(noff, ng, v) << lbits) | (uint64_t)l;
        vals[v] = (uint32_t)v;
    }
}

// perm (new -> old) to inv (old -> new) and the original graph-local id of every new row
__global__ void k_order_maps(int32_t n, const uint32_t* __restrict__ perm, const int32_t* __restrict__ noff,
                             int ng, int32_t* __restrict__ inv, int32_t* __restrict__ orig_local) {
    for (int64_t r = (int64_t)blockIdx.x * kBlock + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * kBlock) {
        const int32_t old = (int32_t)perm[r];
        inv[old] = (int32_t)r;
        orig_local[r] = old - noff[seg_of(noff, ng, old)];
    }
}

__global__ void k_relabel(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                          const int32_t* __restrict__ inv, int32_t* __restrict__ u2,
                          int32_t* __restrict__ v2) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock) {
        u2[e] = inv[eu[e]];
        v2[e] = inv[ev[e]];
    }
}

__global__ void k_invert(int64_t m, const int32_t* __restrict__ f, int32_t* __restrict__ finv) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock)
        finv[f[e]] = (int32_t)e;
}

__global__ void k_gather_ids(int64_t k, const int32_t* __restrict__ ids, const int32_t* __restrict__ map,
                             int32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < k;
         i += (int64_t)gridDim.x * kBlock)
        out[i] = map[ids[i]];
}

// mask[map[e]] = src[e]: the forest, written in the original edge order
__global__ void k_scatter_mask(int64_t m, const uint8_t* __restrict__ src, const int32_t* __restrict__ map,
                               uint8_t* __restrict__ mask) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock)
        mask[map[e]] = src[e];
}

int bits_of(int64_t x) {  // bits needed to hold 0 .. x
    int b = 1;
    while (b < 62 && (1ll << b) <= x) ++b;
    return b;
}

template <typename K>
int grid_of(sfg_ctx* ctx, K kernel, int64_t work) {
    return sfg_grid(ctx, (const void*)kernel, kBlock, 0, work);
}

int64_t round_half_up(double x) { return (int64_t)std::floor(x + 0.5); }

struct GraphGuard {
    sfg_graph* g = nullptr;
    ~GraphGuard() { sfg_graph_free(g); }
};

}  // namespace


// The plan of one batch (see the file comment). Device arrays are owned here.
struct sfg_batch {
    int device = -1;
    int ng = 0;
    sfg_params P{};
    int32_t n = 0;
    int64_t m = 0, ncand = 0, k_total = 0;
    sfg_graph* U = nullptr;    // union of the graphs
    sfg_graph* PU = nullptr;   // union of their spanning forests
    int32_t* d_noff = nullptr; // ng + 1 node offsets
    int64_t* d_eoff = nullptr; // ng + 1 edge offsets
    int64_t* d_coff = nullptr; // ng + 1 candidate offsets
    int64_t* d_k = nullptr;    // per-graph budgets
    uint8_t* forest = nullptr; // m: the forests' edges
    int32_t* cand = nullptr;   // ncand candidate ids (union edge ids, ascending, grouped by graph)
    // locality order (NULL without it): the original graph-local id of every union row, the
    // original union edge id of every edge, and the candidates' original ids
    int32_t* orig_local = nullptr;
    int32_t* orig_edge = nullptr;
    int32_t* cand_orig = nullptr;
    std::vector<int64_t> eoff, counts;
    cudaStream_t stream = nullptr;
};

static void batch_free(sfg_batch* b) {
    if (!b) return;
    SfgDeviceGuard guard(b->device);
    sfg_graph_free(b->U);
    sfg_graph_free(b->PU);
    void* ptrs[] = {b->d_noff, b->d_eoff, b->d_coff, b->d_k, b->forest, b->cand,
                    b->orig_local, b->orig_edge, b->cand_orig};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, b->stream);
    delete b;
}

static sfg_status check_batch_params(sfg_ctx* ctx, const sfg_params* P) {
    if (P->levels != 0)
        return sfg_fail(ctx, SFG_EUNSUPPORTED, "the batched form is flat (levels = 0)");
    if (!sfg_k_supported(P->K, P->storage))
        return sfg_fail(ctx, SFG_EUNSUPPORTED, "K=%d unsupported for dtype %d", P->K, (int)P->storage);
    if (P->smoother != SFG_SMOOTH_JACOBI)
        return sfg_fail(ctx, SFG_EUNSUPPORTED, "the batched form uses the Jacobi smoother only");
    if (P->steps < 0 || !(P->omega > 0.0 && P->omega <= 1.0) || !(P->budget_frac >= 0.0) ||
        (P->budget_unit != 0 && P->budget_unit != 1) ||
        (P->mode != SFG_SCORE_RATIO && P->mode != SFG_SCORE_G && P->mode != SFG_SCORE_P))
        return sfg_fail(ctx, SFG_EINVAL, "invalid sfg_params");
    return SFG_OK;
}

// Breadth-first renumbering of the union (see the file comment): b->U is replaced by its
// relabelled copy; f2c receives the new id of every original union edge.
constexpr int32_t kMaxLevels = 4096;
static sfg_status batch_reorder(sfg_ctx* ctx, sfg_batch* b, int32_t* f2c) {
    const int32_t n = b->n;
    const int64_t m = b->m;
    const int ng = b->ng;
    Scratch s(ctx);
    int32_t *level, *roots, *inv, *u2, *v2;
    unsigned long long* best;
    int* flag;
    uint64_t *keys, *keys2;
    uint32_t *vals, *vals2;
    SFG_TRY(s.get(&level, n));
    SFG_TRY(s.get(&roots, ng));
    SFG_TRY(s.get(&best, ng));
    SFG_TRY(s.get(&flag, 1));
    SFG_TRY(s.get(&keys, n));
    SFG_TRY(s.get(&keys2, n));
    SFG_TRY(s.get(&vals, n));
    SFG_TRY(s.get(&vals2, n));
    SFG_TRY(s.get(&inv, n));
    SFG_TRY(s.get(&u2, m));
    SFG_TRY(s.get(&v2, m));
    int* hflag = nullptr;
    SFG_TRY(sfg_host_word(ctx, 3, &hflag));
    const sfg_graph* U = b->U;
    const int gn = grid_of(ctx, k_bfs_step, n), gg = grid_of(ctx, k_bfs_seed, ng);
    int32_t depth = 0;
    // two searches: the second starts from the farthest node the first reached in each graph
    for (int pass = 0; pass < 2; ++pass) {
        SFG_CUDA(ctx, cudaMemsetAsync(level, 0xff, 4 * (size_t)n, ctx->stream));
        k_bfs_seed<<<gg, kBlock, 0, ctx->stream>>>(ng, b->d_noff, pass ? roots : nullptr, level);
        ++ctx->launches;
        // one launch and one synchronisation per level: the search stops after kMaxLevels levels
        // (nodes further out keep their input order, after the labelled ones)
        for (depth = 0; depth + 1 < kMaxLevels; ++depth) {
            SFG_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
            k_bfs_step<<<gn, kBlock, 0, ctx->stream>>>(n, U->row_ptr, U->colval, depth, level, flag);
            ++ctx->launches;
            SFG_CUDA(ctx, cudaMemcpyAsync(hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            if (!*hflag) break;
        }
        if (pass == 0) {
            SFG_CUDA(ctx, cudaMemsetAsync(best, 0, 8 * (size_t)ng, ctx->stream));
            k_bfs_far<<<gn, kBlock, 0, ctx->stream>>>(n, b->d_noff, ng, level, best);
            k_bfs_roots<<<gg, kBlock, 0, ctx->stream>>>(ng, best, b->d_noff, roots);
            ctx->launches += 2;
        }
        SFG_LAUNCH_CHECK(ctx, "breadth-first search");
    }
    // stable sort of the nodes by (graph, level): depth is the deepest level
    const int lbits = bits_of((int64_t)depth + 1);
    k_order_keys<<<gn, kBlock, 0, ctx->stream>>>(n, b->d_noff, ng, level, depth + 1, lbits, keys, vals);
    ++ctx->launches;
    SFG_TRY(sfg_radix_sort_pairs(ctx, &keys, &vals, &keys2, &vals2, n, lbits + bits_of(ng)));
    SFG_TRY(sfg_alloc(ctx, (void**)&b->orig_local, 4 * (size_t)n + 16));
    k_order_maps<<<gn, kBlock, 0, ctx->stream>>>(n, vals, b->d_noff, ng, inv, b->orig_local);
    ++ctx->launches;
    // the relabelled union, canonicalised again; f2c maps old edge ids to new ones
    sfg_graph* U2 = nullptr;
    if (m > 0) {
        k_relabel<<<grid_of(ctx, k_relabel, m), kBlock, 0, ctx->stream>>>(m, U->eu, U->ev, inv, u2, v2);
        ++ctx->launches;
    }
    SFG_LAUNCH_CHECK(ctx, "locality order");
    SFG_TRY(sfg_build_graph(ctx, n, m, u2, v2, U->ew, false, &U2, f2c));
    if (U2->m != m) {
        sfg_graph_free(U2);
        return sfg_fail(ctx, SFG_EINVAL, "relabelled union lost edges");
    }
    SFG_TRY(sfg_alloc(ctx, (void**)&b->orig_edge, 4 * (size_t)m + 16));
    if (m > 0) {
        k_invert<<<grid_of(ctx, k_invert, m), kBlock, 0, ctx->stream>>>(m, f2c, b->orig_edge);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_invert");
    }
    sfg_graph_free(b->U);
    b->U = U2;
    return SFG_OK;
}

static sfg_status batch_build(sfg_ctx* ctx, int ng, const sfg_graph* const* gs, const sfg_params* P,
                              int flags, sfg_batch* b) {
    const bool autotune = (flags & SFG_BATCH_AUTOTUNE) != 0;
    const bool locality = (flags & SFG_BATCH_LOCALITY) != 0;
    b->device = ctx->device;
    b->stream = ctx->stream;
    b->ng = ng;
    b->P = *P;
    std::vector<int32_t> noff(ng + 1, 0);
    std::vector<int64_t>& eoff = b->eoff;
    eoff.assign(ng + 1, 0);
    std::vector<GDesc> desc(ng);
    for (int g = 0; g < ng; ++g) {
        const sfg_graph* G = gs[g];
        if (!G) return sfg_fail(ctx, SFG_EINVAL, "graph %d is NULL", g);
        if (G->device != ctx->device) return sfg_fail(ctx, SFG_EINVAL, "graph %d is on another device", g);
        if ((int64_t)noff[g] + G->n >= (1ll << 31) || 2 * (eoff[g] + G->m) >= (1ll << 31))
            return sfg_fail(ctx, SFG_EINVAL, "batch too large for int32 indices");
        noff[g + 1] = noff[g] + G->n;
        eoff[g + 1] = eoff[g] + G->m;
        desc[g] = GDesc{G->eu, G->ev, G->ew, G->row_ptr, G->colval, G->eid, G->deg, G->invdeg,
                        noff[g], eoff[g]};
    }
    const int32_t n = noff[ng];
    const int64_t m = eoff[ng];
    b->n = n;
    b->m = m;
    Scratch s(ctx);
    GDesc* d_desc;
    unsigned long long* d_cnt;
    SFG_TRY(s.get(&d_desc, ng));
    SFG_TRY(s.get(&d_cnt, ng));
    SFG_TRY(sfg_alloc(ctx, (void**)&b->d_noff, 4 * (size_t)(ng + 1)));
    SFG_TRY(sfg_alloc(ctx, (void**)&b->d_eoff, 8 * (size_t)(ng + 1)));
    SFG_TRY(sfg_alloc(ctx, (void**)&b->d_coff, 8 * (size_t)(ng + 1)));
    SFG_TRY(sfg_alloc(ctx, (void**)&b->d_k, 8 * (size_t)ng));
    SFG_TRY(sfg_alloc(ctx, (void**)&b->forest, (size_t)m + 16));
    SFG_CUDA(ctx, cudaMemcpyAsync(d_desc, desc.data(), sizeof(GDesc) * ng, cudaMemcpyHostToDevice, ctx->stream));
    SFG_CUDA(ctx, cudaMemcpyAsync(b->d_noff, noff.data(), 4 * (ng + 1), cudaMemcpyHostToDevice, ctx->stream));
    SFG_CUDA(ctx, cudaMemcpyAsync(b->d_eoff, eoff.data(), 8 * (ng + 1), cudaMemcpyHostToDevice, ctx->stream));

    // the disjoint union U
    SFG_TRY(sfg_alloc_graph(ctx, n, m, &b->U));
    if (m > 0) {
        k_union_edges<<<grid_of(ctx, k_union_edges, m), kBlock, 0, ctx->stream>>>(
            m, d_desc, ng, b->d_eoff, b->U->eu, b->U->ev, b->U->ew);
        k_union_entries<<<grid_of(ctx, k_union_entries, 2 * m), kBlock, 0, ctx->stream>>>(
            m, d_desc, ng, b->d_eoff, b->U->colval, b->U->eid);
        ctx->launches += 2;
    }
    k_union_rows<<<grid_of(ctx, k_union_rows, (int64_t)n + 1), kBlock, 0, ctx->stream>>>(
        n, m, d_desc, ng, b->d_noff, b->U->row_ptr, b->U->deg, b->U->invdeg);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_union");

    // locality order: the plan continues on the relabelled union
    int32_t* f2c = nullptr;
    if (locality && n > 0) {
        SFG_TRY(s.get(&f2c, m + 1));
        SFG_TRY(batch_reorder(ctx, b, f2c));
    }

    // spanning forests of every graph, per-graph forest sizes (weight ties broken by original id)
    int64_t n_tree = 0;
    SFG_TRY(sfg_mst_impl(ctx, b->U, nullptr, b->forest, &n_tree, nullptr, b->orig_edge,
                         b->orig_edge ? f2c : nullptr));
    std::vector<int64_t> tree(ng, 0);
    SFG_CUDA(ctx, cudaMemsetAsync(d_cnt, 0, 8 * ng, ctx->stream));
    if (m > 0) {
        k_seg_count<<<grid_of(ctx, k_seg_count, m), kBlock, 0, ctx->stream>>>(m, b->forest, ng,
                                                                            b->d_eoff, d_cnt);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_seg_count");
    }
    SFG_CUDA(ctx, cudaMemcpyAsync(tree.data(), d_cnt, 8 * ng, cudaMemcpyDeviceToHost, ctx->stream));
    SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));

    // per-graph budgets (each graph's P starts as its forest: no edge is over budget)
    std::vector<int64_t> kk(ng), coff(ng + 1, 0);
    b->counts.assign(ng, 0);
    for (int g = 0; g < ng; ++g) {
        const int64_t ng_n = noff[g + 1] - noff[g], ng_m = eoff[g + 1] - eoff[g];
        const int64_t nc = ng_m - tree[g];
        const int64_t base = P->budget_unit == 0 ? ng_n : nc;
        int64_t k = round_half_up(P->budget_frac * (double)base);
        if (k < 0) k = 0;
        if (k > nc) k = nc;
        kk[g] = k;
        b->k_total += k;
        coff[g + 1] = coff[g] + nc;
        b->counts[g] = tree[g] + k;
    }
    b->ncand = coff[ng];
    SFG_CUDA(ctx, cudaMemcpyAsync(b->d_coff, coff.data(), 8 * (ng + 1), cudaMemcpyHostToDevice, ctx->stream));
    SFG_CUDA(ctx, cudaMemcpyAsync(b->d_k, kk.data(), 8 * ng, cudaMemcpyHostToDevice, ctx->stream));
    if (b->k_total > 0) {
        uint8_t* flag;
        int64_t* pos;
        SFG_TRY(s.get(&flag, m));
        SFG_TRY(s.get(&pos, m + 1));
        SFG_TRY(sfg_alloc(ctx, (void**)&b->cand, 4 * (size_t)b->ncand + 16));
        k_not<<<grid_of(ctx, k_not, m), kBlock, 0, ctx->stream>>>(m, b->forest, flag);
        ++ctx->launches;
        SFG_TRY(sfg_scan_u8(ctx, flag, pos, m));
        k_compact<<<grid_of(ctx, k_compact, m), kBlock, 0, ctx->stream>>>(m, flag, pos, b->cand);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_compact");
        if (b->orig_edge) {  // the candidates under their original ids, for the selection
            SFG_TRY(sfg_alloc(ctx, (void**)&b->cand_orig, 4 * (size_t)b->ncand + 16));
            k_gather_ids<<<grid_of(ctx, k_gather_ids, b->ncand), kBlock, 0, ctx->stream>>>(
                b->ncand, b->cand, b->orig_edge, b->cand_orig);
            ++ctx->launches;
            SFG_LAUNCH_CHECK(ctx, "k_gather_ids");
        }
        SFG_TRY(sfg_subgraph_impl(ctx, b->U, b->forest, &b->PU));
        // one-time per-graph structures the sweeps use, built here so that runs never synchronise
        SFG_TRY(sfg_heavy_prepare(ctx, b->U));
        SFG_TRY(sfg_heavy_prepare(ctx, b->PU));
        if (autotune) {
            SFG_TRY(sfg_autotune_impl(ctx, b->U, P->K, P->storage, nullptr, nullptr));
            SFG_TRY(sfg_autotune_impl(ctx, b->PU, P->K, P->storage, nullptr, nullptr));
        }
    }
    SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SFG_OK;
}

// The numeric part: forest copied into mask (m entries, union edge order), then the top-scored
// candidates of every graph added. Launches and stream-ordered allocations only.
static sfg_status batch_run(sfg_ctx* ctx, const sfg_batch* b, uint64_t seed, uint8_t* mask) {
    if (b->m > 0 && b->orig_edge) {
        k_scatter_mask<<<grid_of(ctx, k_scatter_mask, b->m), kBlock, 0, ctx->stream>>>(
            b->m, b->forest, b->orig_edge, mask);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_scatter_mask");
    } else if (b->m > 0) {
        SFG_CUDA(ctx, cudaMemcpyAsync(mask, b->forest, (size_t)b->m, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (b->k_total == 0) return SFG_OK;
    Scratch s(ctx);
    int32_t* sel;
    float* scores;
    SFG_TRY(s.get(&scores, b->ncand));
    SFG_TRY(s.get(&sel, b->k_total));
    const sfg_params& P = b->P;
    SFG_TRY(sfg_filter_score_batched_impl(ctx, b->U, b->PU, b->orig_local, b->ng, b->d_noff, P.K,
                                          P.steps, P.omega, seed, P.storage, b->cand, b->ncand,
                                          P.mode, scores));
    // selection under original edge ids (ties and the output order as without the reordering)
    SFG_TRY(sfg_topk_segmented_impl(ctx, scores, b->cand_orig ? b->cand_orig : b->cand, b->ncand,
                                    b->ng, b->d_coff, b->d_k, b->k_total, sel));
    k_mark<<<grid_of(ctx, k_mark, b->k_total), kBlock, 0, ctx->stream>>>(b->k_total, sel, mask);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_mark");
    return SFG_OK;
}

extern "C" {

sfg_status sfg_batch_create(sfg_ctx* ctx, int ng, const sfg_graph* const* gs, const sfg_params* P,
                            int flags, sfg_batch** out) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!out) return sfg_fail(ctx, SFG_EINVAL, "out is NULL");
    *out = nullptr;
    if (ng < 1 || !gs || !P) return sfg_fail(ctx, SFG_EINVAL, "bad batch arguments");
    SFG_TRY(check_batch_params(ctx, P));
    sfg_batch* b = new sfg_batch();
    if (flags & ~(SFG_BATCH_AUTOTUNE | SFG_BATCH_LOCALITY)) {
        delete b;
        return sfg_fail(ctx, SFG_EINVAL, "unknown batch flags %d", flags);
    }
    const sfg_status st = batch_build(ctx, ng, gs, P, flags, b);
    if (st != SFG_OK) {
        batch_free(b);
        return st;
    }
    *out = b;
    return SFG_OK;
}

sfg_status sfg_batch_info(const sfg_batch* b, int* ng_host, int64_t* edges_host,
                          int64_t* edge_offsets_host, int64_t* n_selected_host) {
    if (!b) return SFG_EINVAL;
    if (ng_host) *ng_host = b->ng;
    if (edges_host) *edges_host = b->m;
    if (edge_offsets_host)
        for (int g = 0; g <= b->ng; ++g) edge_offsets_host[g] = b->eoff[(size_t)g];
    if (n_selected_host)
        for (int g = 0; g < b->ng; ++g) n_selected_host[g] = b->counts[(size_t)g];
    return SFG_OK;
}

sfg_status sfg_batch_run(sfg_ctx* ctx, const sfg_batch* b, uint64_t seed, uint8_t* mask_out) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!b) return sfg_fail(ctx, SFG_EINVAL, "batch is NULL");
    if (b->device != ctx->device) return sfg_fail(ctx, SFG_EINVAL, "batch is on another device");
    if (b->m == 0) return SFG_OK;
    SFG_TRY(sfg_check_dev(ctx, mask_out, "mask_out"));
    return batch_run(ctx, b, seed, mask_out);
}

void sfg_batch_destroy(sfg_batch* b) { batch_free(b); }

sfg_status sfg_sparsify_batched(sfg_ctx* ctx, int ng, const sfg_graph* const* gs,
                                const sfg_params* P, uint8_t* const* masks_out,
                                int64_t* n_selected_host) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (ng < 1 || !gs || !P || !masks_out) return sfg_fail(ctx, SFG_EINVAL, "bad batch arguments");
    SFG_TRY(check_batch_params(ctx, P));
    for (int g = 0; g < ng; ++g)
        if (gs[g] && gs[g]->m > 0) SFG_TRY(sfg_check_dev(ctx, masks_out[g], "masks_out[g]"));
    sfg_batch* b = new sfg_batch();
    struct Owner { sfg_batch* b; ~Owner() { batch_free(b); } } owner{b};
    SFG_TRY(batch_build(ctx, ng, gs, P, 0, b));
    Scratch s(ctx);
    uint8_t* mask;
    uint8_t** d_outs;
    SFG_TRY(s.get(&mask, b->m));
    SFG_TRY(s.get(&d_outs, ng));
    SFG_CUDA(ctx, cudaMemcpyAsync(d_outs, masks_out, sizeof(uint8_t*) * ng, cudaMemcpyHostToDevice, ctx->stream));
    SFG_TRY(batch_run(ctx, b, P->seed, mask));
    if (b->m > 0) {
        k_split<<<grid_of(ctx, k_split, b->m), kBlock, 0, ctx->stream>>>(b->m, mask, ng, b->d_eoff, d_outs);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_split");
    }
    SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // d_outs' host source goes out of scope
    if (n_selected_host)
        for (int g = 0; g < ng; ++g) n_selected_host[g] = b->counts[(size_t)g];
    return SFG_OK;
}

}  // extern "C"
