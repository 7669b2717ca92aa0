// The whole method (Algorithm 1), orchestrated on the host over the device kernels.
//
// Flat: maximum spanning forest of G, then one round of edge recovery: embed G and the current
// sparsifier P from the same seed, score every edge of G outside P, add the top ones. Multilevel:
// coarsen `levels` times (caching each level's embedding), sparsify the coarsest graph flat, then
// for each finer level map the sparsifier back and run edge recovery there with the cached
// embedding of G_l.
#include <cmath>

#include "sfg_internal.cuh"

namespace {

constexpr int kBlock = 256;

__global__ void k_not_mask(int64_t m, const uint8_t* __restrict__ mask, uint8_t* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock)
        out[e] = mask[e] == 0;
}

__global__ void k_compact_ids(int64_t m, const uint8_t* __restrict__ flag,
                              const int64_t* __restrict__ pos, int32_t* __restrict__ ids) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock)
        if (flag[e]) ids[pos[e]] = (int32_t)e;
}

__global__ void k_f32_to_bf16(int64_t n, const float* __restrict__ x, __nv_bfloat16* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kBlock)
        y[i] = __float2bfloat16_rn(x[i]);
}

__global__ void k_set_mask(int64_t k, const int32_t* __restrict__ ids, uint8_t* __restrict__ mask) {
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < k;
         i += (int64_t)gridDim.x * kBlock)
        mask[ids[i]] = 1;
}

// Smoother choice and its omega range: weighted Jacobi (0, 1], Gauss-Seidel / SOR (0, 2).
bool omega_ok(const sfg_params* P) {
    if (P->smoother == SFG_SMOOTH_JACOBI) return P->omega > 0.0 && P->omega <= 1.0;
    if (P->smoother == SFG_SMOOTH_GAUSS_SEIDEL) return P->omega > 0.0 && P->omega < 2.0;
    return false;
}

sfg_status smooth_any(sfg_ctx* ctx, const sfg_params* P, const sfg_graph* g, uint64_t seed,
                      sfg_dtype storage, void* x) {
    if (P->smoother == SFG_SMOOTH_GAUSS_SEIDEL)
        return sfg_smooth_gs_impl(ctx, g, P->K, P->steps, P->omega, seed, storage, x);
    return sfg_smooth_impl(ctx, g, P->K, P->steps, P->omega, seed, storage, x);
}

uint64_t level_seed(uint64_t seed, int l) { return l == 0 ? seed : sfg_splitmix64(seed ^ (uint64_t)l); }

int64_t round_half_up(double x) { return (int64_t)std::floor(x + 0.5); }

size_t elem_size(sfg_dtype dt) { return dt == SFG_BF16 ? 2 : 4; }

// Edge recovery at one level (Sec. 3.5; the embedding, scoring and selection steps of
// Algorithm 1). `mask` holds the current sparsifier of g and receives the added edges. XG_f32: the
// FP32 embedding of g from this level's seed, cached from coarsening (may be NULL: computed here
// in the requested storage).
sfg_status recover(sfg_ctx* ctx, const sfg_graph* g, const sfg_params* P, uint64_t seed,
                   int64_t forest, const float* XG_f32, uint8_t* mask) {
    const int64_t m = g->m;
    const int64_t base = P->budget_unit == 0 ? (int64_t)g->n : m - forest;
    const int64_t target = round_half_up(P->budget_frac * (double)base);
    int64_t in_p = 0;
    SFG_TRY(sfg_count_mask(ctx, mask, m, &in_p));
    const int64_t ncand = m - in_p;
    int64_t k = target - (in_p - forest);
    if (k < 0) k = 0;
    if (k > ncand) k = ncand;
    if (k == 0) return SFG_OK;

    Scratch s(ctx);
    uint8_t* flag;
    int64_t* pos;
    int32_t *cand, *sel;
    float* scores;
    SFG_TRY(s.get(&flag, m));
    SFG_TRY(s.get(&pos, m + 1));
    SFG_TRY(s.get(&cand, ncand));
    SFG_TRY(s.get(&scores, ncand));
    SFG_TRY(s.get(&sel, k));
    const int gm = sfg_grid(ctx, (const void*)k_not_mask, kBlock, 0, m);
    k_not_mask<<<gm, kBlock, 0, ctx->stream>>>(m, mask, flag); ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_not_mask");
    SFG_TRY(sfg_scan_u8(ctx, flag, pos, m));
    k_compact_ids<<<gm, kBlock, 0, ctx->stream>>>(m, flag, pos, cand); ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_compact_ids");

    sfg_graph* pg = nullptr;
    SFG_TRY(sfg_subgraph_impl(ctx, g, mask, &pg));
    struct Guard { sfg_graph* g; ~Guard() { sfg_graph_free(g); } } guard{pg};

    if (P->smoother == SFG_SMOOTH_GAUSS_SEIDEL) {  // the paper's smoother: embed both, then score
        // P sweeps in G's colour order (a proper colouring of P as well): no second colouring
        SFG_TRY(sfg_gs_inherit(ctx, pg, g));
        const size_t blk = (size_t)g->n * P->K * elem_size(P->storage);
        void* xp;
        const void* xg = XG_f32;
        SFG_TRY(s.get((char**)&xp, blk));
        if (!xg || P->storage != SFG_F32) {
            void* x;
            SFG_TRY(s.get((char**)&x, blk));
            SFG_TRY(sfg_smooth_gs_impl(ctx, g, P->K, P->steps, P->omega, seed, P->storage, x));
            xg = x;
        }
        SFG_TRY(sfg_smooth_gs_impl(ctx, pg, P->K, P->steps, P->omega, seed, P->storage, xp));
        SFG_TRY(sfg_score_impl(ctx, g, xg, xp, P->K, P->storage, cand, ncand, P->mode, scores));
    } else if (!XG_f32) {  // embed G and P from one seeded block and score in one pass
        SFG_TRY(sfg_filter_score_impl(ctx, g, pg, P->K, P->steps, P->omega, seed, P->storage, cand,
                                      ncand, P->mode, scores));
    } else {  // reuse the level's cached FP32 embedding of G (rounded once for BF16 storage)
        const size_t blk = (size_t)g->n * P->K * elem_size(P->storage);
        void* xp;
        SFG_TRY(s.get((char**)&xp, blk));
        const void* xg = XG_f32;
        if (P->storage != SFG_F32) {
            void* x;
            SFG_TRY(s.get((char**)&x, blk));
            const int64_t cnt = (int64_t)g->n * P->K;
            k_f32_to_bf16<<<sfg_grid(ctx, (const void*)k_f32_to_bf16, kBlock, 0, cnt), kBlock, 0,
                            ctx->stream>>>(cnt, XG_f32, (__nv_bfloat16*)x);
            ++ctx->launches;
            SFG_LAUNCH_CHECK(ctx, "k_f32_to_bf16");
            xg = x;
        }
        SFG_TRY(sfg_smooth_impl(ctx, pg, P->K, P->steps, P->omega, seed, P->storage, xp));
        SFG_TRY(sfg_score_impl(ctx, g, xg, xp, P->K, P->storage, cand, ncand, P->mode, scores));
    }
    SFG_TRY(sfg_topk_impl(ctx, scores, cand, ncand, k, sel));
    k_set_mask<<<sfg_grid(ctx, (const void*)k_set_mask, kBlock, 0, k), kBlock, 0, ctx->stream>>>(
        k, sel, mask); ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_set_mask");
    return SFG_OK;
}

struct Level {
    sfg_graph* g = nullptr;   // G_l (level 0 borrowed)
    int32_t* agg = nullptr;   // map G_{l-1} -> G_l (l >= 1)
    int32_t* f2c = nullptr;   // fine edge of G_{l-1} -> edge of G_l
    float* xg = nullptr;      // FP32 embedding of G_l used for coarsening (l < lf)
    uint8_t* pmask = nullptr; // the level's sparsifier P_l over G_l's edges
};

}  // namespace

// The coarsening hierarchy of one sfg_sparsify call (Algorithm 1's [G_1 .. G_lf; H_1 .. H_lf]
// with each level's sparsifier): device arrays owned here, freed by sfg_hierarchy_destroy.
struct sfg_hierarchy {
    int device = -1;
    cudaStream_t stream = nullptr;
    const sfg_graph* g0 = nullptr;        // the input graph (borrowed)
    std::vector<Level> lv;                // levels 0..lf (level 0's graph is g0)
};

static void hierarchy_free(sfg_hierarchy* h) {
    if (!h) return;
    SfgDeviceGuard guard(h->device);
    for (size_t l = 0; l < h->lv.size(); ++l) {
        Level& v = h->lv[l];
        if (l > 0) sfg_graph_free(v.g);
        void* ptrs[] = {v.agg, v.f2c, v.pmask};
        for (void* p : ptrs)
            if (p) cudaFreeAsync(p, h->stream);
    }
    delete h;
}

extern "C" sfg_status sfg_sparsify(sfg_ctx* ctx, const sfg_graph* G, const sfg_params* P,
                                   uint8_t* mask_out, int64_t* n_selected_host,
                                   sfg_hierarchy** hier_out) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (hier_out) *hier_out = nullptr;
    if (!G || !P) return sfg_fail(ctx, SFG_EINVAL, "NULL argument");
    if (!sfg_k_supported(P->K, P->storage) || (P->levels > 0 && !sfg_k_supported(P->K, SFG_F32)))
        return sfg_fail(ctx, SFG_EUNSUPPORTED, "K=%d unsupported for dtype %d", P->K,
                        (int)P->storage);
    if (P->steps < 0 || P->levels < 0 || !omega_ok(P) ||
        !(P->budget_frac >= 0.0) || (P->budget_unit != 0 && P->budget_unit != 1) ||
        (P->mode != SFG_SCORE_RATIO && P->mode != SFG_SCORE_G && P->mode != SFG_SCORE_P))
        return sfg_fail(ctx, SFG_EINVAL, "invalid sfg_params");
    if (G->m > 0) SFG_TRY(sfg_check_dev(ctx, mask_out, "mask_out"));

    // The levels live in a hierarchy object; it goes to the caller when asked for (and on
    // success), else it is freed on return.
    sfg_hierarchy* h = new sfg_hierarchy();
    h->device = ctx->device;
    h->stream = ctx->stream;
    h->g0 = G;
    h->lv.resize(1);
    h->lv[0].g = const_cast<sfg_graph*>(G);
    struct Owner {
        sfg_hierarchy* h;
        ~Owner() { hierarchy_free(h); }
    } owner{h};
    std::vector<Level>& lv = h->lv;
    Scratch s(ctx);

    // Algorithm 1, coarsening phase: multilevel spectral graph reduction. The aggregation (an
    // argmin decided by floating point) is taken on FP32 embeddings whatever the storage of the
    // edge-recovery blocks, so BF16 storage changes only the recovery scores, not the hierarchy.
    for (int l = 1; l <= P->levels; ++l) {
        if (lv.back().g->m == 0) break;
        {
            Level& f = lv.back();
            SFG_TRY(s.get(&f.xg, (size_t)f.g->n * P->K));
            SFG_TRY(smooth_any(ctx, P, f.g, level_seed(P->seed, l - 1), SFG_F32, f.xg));
        }
        lv.emplace_back();
        Level& f = lv[lv.size() - 2];
        Level& c = lv.back();
        SFG_TRY(sfg_alloc(ctx, (void**)&c.agg, (size_t)f.g->n * 4 + 16));
        SFG_TRY(sfg_alloc(ctx, (void**)&c.f2c, (size_t)f.g->m * 4 + 16));
        int32_t nc = 0;
        SFG_TRY(sfg_coarsen_impl(ctx, f.g, f.xg, P->K, SFG_F32, c.agg, c.f2c, &nc, &c.g));
    }
    const int lf = (int)lv.size() - 1;

    // coarsest level: spanning forest + recovered off-tree edges
    const sfg_graph* gc = lv[lf].g;
    SFG_TRY(sfg_alloc(ctx, (void**)&lv[lf].pmask, (size_t)gc->m + 16));
    uint8_t* pm = lv[lf].pmask;
    int64_t n_tree = 0;
    SFG_TRY(sfg_mst_impl(ctx, gc, nullptr, pm, &n_tree));
    const int64_t comps = (int64_t)gc->n - n_tree;  // same at every level: aggregates are connected
    SFG_TRY(recover(ctx, gc, P, level_seed(P->seed, lf), n_tree, nullptr, pm));

    // Algorithm 1, level loop: map back and recover edges level by level
    for (int l = lf; l >= 1; --l) {
        const sfg_graph* f = lv[l - 1].g;
        SFG_TRY(sfg_alloc(ctx, (void**)&lv[l - 1].pmask, (size_t)f->m + 16));
        uint8_t* pf = lv[l - 1].pmask;
        SFG_TRY(sfg_backward_impl(ctx, f, lv[l].agg, lv[l].f2c, lv[l].g, pm, pf));
        SFG_TRY(recover(ctx, f, P, level_seed(P->seed, l - 1), (int64_t)f->n - comps, lv[l - 1].xg,
                        pf));
        pm = pf;
    }
    for (Level& v : lv) v.xg = nullptr;  // scratch, freed with s
    if (G->m > 0)
        SFG_CUDA(ctx, cudaMemcpyAsync(mask_out, pm, G->m, cudaMemcpyDeviceToDevice, ctx->stream));
    if (n_selected_host) SFG_TRY(sfg_count_mask(ctx, mask_out, G->m, n_selected_host));
    if (hier_out) {
        *hier_out = h;
        owner.h = nullptr;
    }
    return SFG_OK;
}

extern "C" {

sfg_status sfg_hierarchy_levels(const sfg_hierarchy* h, int* levels_host) {
    if (!h || !levels_host) return SFG_EINVAL;
    *levels_host = (int)h->lv.size() - 1;
    return SFG_OK;
}

sfg_status sfg_hierarchy_graph(const sfg_hierarchy* h, int level, const sfg_graph** out) {
    if (!h || !out || level < 0 || level >= (int)h->lv.size()) return SFG_EINVAL;
    *out = h->lv[(size_t)level].g;
    return SFG_OK;
}

sfg_status sfg_hierarchy_map(sfg_ctx* ctx, const sfg_hierarchy* h, int level, int32_t* agg_out,
                             int32_t* fine2coarse_out) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!h || level < 1 || level >= (int)h->lv.size())
        return sfg_fail(ctx, SFG_EINVAL, "level must be in [1, levels]");
    const Level& c = h->lv[(size_t)level];
    const sfg_graph* f = h->lv[(size_t)level - 1].g;
    if (agg_out && f->n > 0) {
        SFG_TRY(sfg_check_dev(ctx, agg_out, "agg_out"));
        SFG_CUDA(ctx, cudaMemcpyAsync(agg_out, c.agg, (size_t)f->n * 4, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
    }
    if (fine2coarse_out && f->m > 0) {
        SFG_TRY(sfg_check_dev(ctx, fine2coarse_out, "fine2coarse_out"));
        SFG_CUDA(ctx, cudaMemcpyAsync(fine2coarse_out, c.f2c, (size_t)f->m * 4,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return SFG_OK;
}

sfg_status sfg_hierarchy_mask(sfg_ctx* ctx, const sfg_hierarchy* h, int level, uint8_t* mask_out) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!h || level < 0 || level >= (int)h->lv.size())
        return sfg_fail(ctx, SFG_EINVAL, "level must be in [0, levels]");
    const Level& v = h->lv[(size_t)level];
    if (v.g->m == 0) return SFG_OK;
    SFG_TRY(sfg_check_dev(ctx, mask_out, "mask_out"));
    SFG_CUDA(ctx, cudaMemcpyAsync(mask_out, v.pmask, (size_t)v.g->m, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    return SFG_OK;
}

void sfg_hierarchy_destroy(sfg_hierarchy* h) { hierarchy_free(h); }

}  // extern "C"

extern "C" sfg_status sfg_sparsify_learned(sfg_ctx* ctx, const sfg_graph* G, const sfg_params* P,
                                           const sfg_mlp* net, int feat_steps, double propose_frac,
                                           uint8_t* mask_out, int64_t* n_selected_host) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!G || !P) return sfg_fail(ctx, SFG_EINVAL, "NULL argument");
    if (P->levels != 0) return sfg_fail(ctx, SFG_EUNSUPPORTED, "learned proposals are flat (levels = 0)");
    if (P->smoother != SFG_SMOOTH_JACOBI)
        return sfg_fail(ctx, SFG_EUNSUPPORTED, "learned proposals use the Jacobi smoother only");
    if (!net || !(propose_frac < 1.0)) return sfg_sparsify(ctx, G, P, mask_out, n_selected_host, nullptr);
    if (!sfg_k_supported(P->K, P->storage))
        return sfg_fail(ctx, SFG_EUNSUPPORTED, "K=%d unsupported for dtype %d", P->K, (int)P->storage);
    if (feat_steps < 0 || !(propose_frac > 0.0) || P->steps < 0 || !(P->omega > 0.0 && P->omega <= 1.0) ||
        !(P->budget_frac >= 0.0) || (P->budget_unit != 0 && P->budget_unit != 1) ||
        (P->mode != SFG_SCORE_RATIO && P->mode != SFG_SCORE_G && P->mode != SFG_SCORE_P))
        return sfg_fail(ctx, SFG_EINVAL, "invalid arguments");
    if (G->m > 0) SFG_TRY(sfg_check_dev(ctx, mask_out, "mask_out"));
    const int64_t m = G->m;
    int64_t n_tree = 0;
    SFG_TRY(sfg_mst_impl(ctx, G, nullptr, mask_out, &n_tree));
    const int64_t ncand = m - n_tree;
    const int64_t base = P->budget_unit == 0 ? (int64_t)G->n : ncand;
    int64_t k = round_half_up(P->budget_frac * (double)base);
    if (k < 0) k = 0;
    if (k > ncand) k = ncand;
    if (k > 0) {
        int64_t nprop = round_half_up(propose_frac * (double)ncand);
        if (nprop < k) nprop = k;
        if (nprop > ncand) nprop = ncand;
        Scratch s(ctx);
        uint8_t* flag;
        int64_t* pos;
        int32_t *cand, *prop, *sel;
        float *feats, *pred, *scores;
        SFG_TRY(s.get(&flag, m));
        SFG_TRY(s.get(&pos, m + 1));
        SFG_TRY(s.get(&cand, ncand));
        SFG_TRY(s.get(&feats, (size_t)ncand * SFG_MLP_NFEAT));
        SFG_TRY(s.get(&pred, ncand));
        SFG_TRY(s.get(&prop, nprop));
        SFG_TRY(s.get(&scores, nprop));
        SFG_TRY(s.get(&sel, k));
        const int gm = sfg_grid(ctx, (const void*)k_not_mask, kBlock, 0, m);
        k_not_mask<<<gm, kBlock, 0, ctx->stream>>>(m, mask_out, flag);
        ++ctx->launches;
        SFG_TRY(sfg_scan_u8(ctx, flag, pos, m));
        k_compact_ids<<<gm, kBlock, 0, ctx->stream>>>(m, flag, pos, cand);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_compact_ids");
        sfg_graph* pg = nullptr;
        SFG_TRY(sfg_subgraph_impl(ctx, G, mask_out, &pg));
        struct Guard { sfg_graph* g; ~Guard() { sfg_graph_free(g); } } guard{pg};
        SFG_TRY(sfg_edge_features_impl(ctx, G, pg, P->K, feat_steps, P->omega, P->seed, P->storage,
                                       cand, ncand, feats));
        SFG_TRY(sfg_mlp_forward_impl(ctx, net, feats, ncand, pred));
        SFG_TRY(sfg_topk_impl(ctx, pred, cand, ncand, nprop, prop));
        SFG_TRY(sfg_filter_score_impl(ctx, G, pg, P->K, P->steps, P->omega, P->seed, P->storage,
                                      prop, nprop, P->mode, scores));
        SFG_TRY(sfg_topk_impl(ctx, scores, prop, nprop, k, sel));
        k_set_mask<<<sfg_grid(ctx, (const void*)k_set_mask, kBlock, 0, k), kBlock, 0, ctx->stream>>>(
            k, sel, mask_out);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_set_mask");
        SFG_TRY(sfg_mlp_check_impl(ctx, net));
    }
    if (n_selected_host) SFG_TRY(sfg_count_mask(ctx, mask_out, m, n_selected_host));
    return SFG_OK;
}

// Sparsification to a target condition number (Sec. 2.2: P is sigma-similar to G when
// kappa(L_G, L_P) <= sigma^2; Sec. 3.4 aims at a desired kappa; Algorithm 1 takes sigma). Flat:
// P starts as the maximum spanning forest; each round measures kappa(L_G, L_P) with the Lanczos
// estimator and stops once it is at most kappa_target, else re-embeds G and the current P from
// the same seed, scores every edge outside P and adds the top ones, so that P holds
// round_half_up(r * batch_frac * base) edges beyond the forest after round r.
extern "C" sfg_status sfg_sparsify_to_kappa(sfg_ctx* ctx, const sfg_graph* G, const sfg_params* P,
                                            double kappa_target, double batch_frac, int max_rounds,
                                            int kappa_steps, uint8_t* mask_out,
                                            int64_t* n_selected_host, double* kappa_trace_host,
                                            int* rounds_host) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!G || !P) return sfg_fail(ctx, SFG_EINVAL, "NULL argument");
    if (!sfg_k_supported(P->K, P->storage))
        return sfg_fail(ctx, SFG_EUNSUPPORTED, "K=%d unsupported for dtype %d", P->K,
                        (int)P->storage);
    if (P->steps < 0 || P->levels != 0 || !omega_ok(P) ||
        (P->budget_unit != 0 && P->budget_unit != 1) ||
        (P->mode != SFG_SCORE_RATIO && P->mode != SFG_SCORE_G && P->mode != SFG_SCORE_P))
        return sfg_fail(ctx, SFG_EINVAL, "invalid sfg_params (levels must be 0)");
    if (!(kappa_target >= 1.0) || !(batch_frac > 0.0) || max_rounds < 0 || kappa_steps < 1)
        return sfg_fail(ctx, SFG_EINVAL, "invalid kappa_target, batch_frac, max_rounds or kappa_steps");
    if (G->m > 0) SFG_TRY(sfg_check_dev(ctx, mask_out, "mask_out"));
    int64_t forest = 0;
    SFG_TRY(sfg_mst_impl(ctx, G, nullptr, mask_out, &forest));
    int r = 0;
    for (;; ++r) {
        double kap = 1.0;
        SFG_TRY(sfg_kappa_impl(ctx, G, mask_out, kappa_steps, P->seed ^ 0x6b617070ull, &kap, nullptr));
        if (kappa_trace_host) kappa_trace_host[r] = kap;
        if (kap <= kappa_target || r == max_rounds) break;
        int64_t before = 0, after = 0;
        SFG_TRY(sfg_count_mask(ctx, mask_out, G->m, &before));
        sfg_params Pr = *P;
        Pr.budget_frac = (double)(r + 1) * batch_frac;
        SFG_TRY(recover(ctx, G, &Pr, P->seed, forest, nullptr, mask_out));
        SFG_TRY(sfg_count_mask(ctx, mask_out, G->m, &after));
        if (after == before) break;  // nothing left to add
    }
    if (rounds_host) *rounds_host = r;
    if (n_selected_host) SFG_TRY(sfg_count_mask(ctx, mask_out, G->m, n_selected_host));
    return SFG_OK;
}
