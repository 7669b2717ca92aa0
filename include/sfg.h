/*
 * sfg.h - C ABI of the GB300 (sm_103a) SF-GRASS hot path.
 *
 * The library computes the data-parallel core of SF-GRASS (Zhang, Zhao, Feng, "SF-GRASS:
 * Solver-Free Graph Spectral Sparsification", ICCAD 2020): the Laplacian of a weighted undirected
 * graph, the local spectral embedding by weighted-Jacobi smoothing of K random vectors, the
 * spectral-perturbation score of candidate edges, top-k edge selection, spanning-tree backbones,
 * one level of spectral coarsening, the sparsifier backward mapping, and the whole flat or
 * multilevel method (Algorithm 1).
 *
 * Conventions shared by every call:
 *  - Pointers are DEVICE pointers (memory of the context's device) unless the name ends in
 *    _host. The caller owns every buffer it passes; opaque objects (sfg_ctx, sfg_graph) are owned
 *    by the library and released by their *_destroy call.
 *  - Every call is ordered on the context's CUDA stream. Calls return as soon as their work is
 *    queued, except where an argument ends in _host or the call's comment says it synchronises.
 *  - Errors are returned as sfg_status, never thrown or aborted; sfg_last_error() holds the text
 *    of the most recent failure on that context. Invalid arguments give SFG_EINVAL and queue no
 *    work; a failing CUDA call gives SFG_ECUDA.
 *  - Results are deterministic for a fixed input, parameters and seed.
 *  - Graph sizes: 1 <= n < 2^31 nodes; at most 2^30 - 1 distinct edges (2m stored entries must
 *    fit an int32).
 */
#ifndef SFG_H
#define SFG_H

#include <stdint.h>

#if defined(__GNUC__)
#define SFG_API __attribute__((visibility("default")))
#else
#define SFG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SFG_OK = 0,
    SFG_EINVAL = 1,       /* bad argument: range, NULL, size, non-finite or non-positive weight */
    SFG_ENOMEM = 2,       /* device allocation failed */
    SFG_ECUDA = 3,        /* a CUDA runtime call failed */
    SFG_ETIMEOUT = 4,     /* an iteration limit ran out before convergence */
    SFG_ECAPACITY = 5,    /* an output buffer is too small */
    SFG_EUNSUPPORTED = 6  /* valid but not implemented (e.g. an unsupported K / dtype pair) */
} sfg_status;

/* Storage type of the N x K vector block. Arithmetic is always FP32 with FP32 accumulation. */
typedef enum { SFG_F32 = 0, SFG_BF16 = 1 } sfg_dtype;

/* Edge score (Sec. 3.5, Eqs. formula_eig_perturb1_conclusion and ..._conclusion2, with the
 * eigenvector block U replaced by the smoothed block X; the scoring and selection steps of Algorithm 1).
 * s_G = w(p,q) * ||X_G^T e_pq||^2 and s_P = w(p,q) * ||X_P^T e_pq||^2, where X_G is the block
 * smoothed on L_G and X_P the block smoothed on L_P from the same seed.
 * RATIO: s_P / (s_G + eta); G: s_G (Algorithm 1 embeds G); P: s_P (Sec. 3.5 perturbs L_P). */
typedef enum { SFG_SCORE_RATIO = 0, SFG_SCORE_G = 1, SFG_SCORE_P = 2 } sfg_score_mode;

typedef struct sfg_ctx sfg_ctx;     /* device, borrowed stream, last error, optional timers */
typedef struct sfg_graph sfg_graph; /* canonical edge list + CSR Laplacian, device-resident */
typedef struct sfg_hierarchy sfg_hierarchy; /* levels of one multilevel run (see sfg_sparsify) */

/* ---------------------------------------------------------------------------------------------
 * Context
 * ------------------------------------------------------------------------------------------- */

/* Create a context on `device` that queues all work on `cuda_stream` (a cudaStream_t; NULL =
 * the legacy default stream). The stream is borrowed: it must outlive the context and every
 * graph created through it. */
SFG_API sfg_status sfg_ctx_create(sfg_ctx** out, int device, void* cuda_stream);
/* Destroys the context and returns the unused memory of the library's pool to the device
 * (graphs and networks made through it stay valid until they are destroyed). */
SFG_API void sfg_ctx_destroy(sfg_ctx* ctx);
/* Device memory: every allocation of the library (graphs, scratch) comes stream-ordered from one
 * pool per device, shared by the contexts on that device and kept for the life of the process,
 * which holds freed memory for reuse instead of returning it at each synchronisation.
 * sfg_ctx_trim synchronises the context stream and returns the pool's unused memory to the
 * device (an allocation that fails also trims and retries once). */
SFG_API sfg_status sfg_ctx_trim(sfg_ctx* ctx);
SFG_API sfg_status sfg_ctx_set_stream(sfg_ctx* ctx, void* cuda_stream);
/* Text of the last error on this context ("" if none). Valid until the next call on ctx. */
SFG_API const char* sfg_last_error(const sfg_ctx* ctx);

/* Optional per-kernel timing: when on, each launch of the library's kernels is bracketed by
 * CUDA events on the context stream. sfg_ctx_kernel_time synchronises the stream and returns,
 * for kernels whose name starts with `prefix`, the number of timed launches and their summed
 * duration in milliseconds. sfg_ctx_timing(ctx, 1) also clears earlier records. */
SFG_API sfg_status sfg_ctx_timing(sfg_ctx* ctx, int on);
SFG_API sfg_status sfg_ctx_kernel_time(sfg_ctx* ctx, const char* prefix, int64_t* launches_host,
                               double* ms_host);

/* Number of kernels this context has launched so far (host counter, no synchronisation). */
SFG_API sfg_status sfg_ctx_launches(const sfg_ctx* ctx, int64_t* launches_host);

/* ---------------------------------------------------------------------------------------------
 * Graph and Laplacian (Sec. 2.1, Eq. formula_adjacency and the definition of D under it;
 * Sec. 4 input convention: positive weights)
 * ------------------------------------------------------------------------------------------- */

/* Build the canonical form and the CSR Laplacian of the weighted undirected graph given by the
 * m input edges (u[i], v[i], w[i]), 0 <= u, v < n, w finite and > 0 (else SFG_EINVAL).
 * Canonical form: each edge stored once with u < v, sorted by (u, v); parallel edges merged by
 * adding their weights (in FP64, in input order, rounded once to FP32); self-loops dropped.
 * Edge id = position in the canonical list. The CSR holds both directions of every edge, each
 * row sorted by column, and the FP64 degrees D(p,p) = sum of the row. Synchronises (reads back
 * the validation flag and the canonical edge count). */
SFG_API sfg_status sfg_laplacian(sfg_ctx* ctx, int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                         const float* w, sfg_graph** out);
SFG_API void sfg_graph_destroy(sfg_graph* g);
SFG_API sfg_status sfg_graph_info(const sfg_graph* g, int32_t* n_host, int64_t* m_host);
/* Copy the canonical edge list (m entries each). */
SFG_API sfg_status sfg_graph_edges(sfg_ctx* ctx, const sfg_graph* g, int32_t* u, int32_t* v, float* w);
/* Copy the CSR: row_ptr[n+1], col[2m], val[2m] (= w), eid[2m] (canonical edge id of each entry),
 * deg[n] (FP64). Any pointer may be NULL to skip that array. */
SFG_API sfg_status sfg_graph_csr(sfg_ctx* ctx, const sfg_graph* g, int32_t* row_ptr, int32_t* col,
                         float* val, int32_t* eid, double* deg);
/* The subgraph P of G made of the edges e with mask[e] != 0 (mask has m entries), same nodes,
 * same weights; its canonical list is G's list filtered in order. Synchronises. */
SFG_API sfg_status sfg_graph_subgraph(sfg_ctx* ctx, const sfg_graph* g, const uint8_t* mask,
                              sfg_graph** out);

/* ---------------------------------------------------------------------------------------------
 * Local spectral embedding (Sec. 3.2: K random vectors orthogonal to the all-one vector, a few
 * relaxation sweeps on L x = 0)
 * ------------------------------------------------------------------------------------------- */

/* X_out (n x K, row-major, `storage`) <- the smoothed, projected block:
 *  1. X0[i,k] = Gaussian entry j = i*K + k of this counter-based generator, rounded to
 *     `storage`; each column's mean removed (FP64 sums). The removed mean is the D-weighted one,
 *     which the sweeps keep: it differs from the plain mean by a constant vector that step 3
 *     removes anyway, so the result is that of the plain reading, without FP32 having to cancel
 *     a persisting constant on fast-mixing graphs. SplitMix64 (Steele, Lea & Flood 2014),
 *     started in state s0 = splitmix64(seed), gives output o_p = splitmix64(s0 + p * gamma) for
 *     the pair of entries 2p, 2p+1: u1 = ((o_p >> 32) + 1) 2^-32, u2 = ((o_p >> 8) mod 2^24)
 *     2^-24, r = sqrt(-2 ln u1), X0_2p = r cos(2 pi u2), X0_2p+1 = r sin(2 pi u2). Evaluated in
 *     FP32 (logf, sincospif), within a few FP32 ulp of the FP64 value.
 *  2. `steps` weighted-Jacobi sweeps X <- X - omega D^-1 L X = (1 - omega) X + omega D^-1 A X
 *     (D^-1 formed in FP64 once per call; rows with D(p,p) = 0 are left unchanged).
 *  3. Projection: each column's mean removed again and the column scaled to unit RMS.
 * K must be one of 4, 8, 16, 32, 64 (SFG_F32) or 8, 16, 32, 64 (SFG_BF16), else
 * SFG_EUNSUPPORTED. 0 < omega <= 1, steps >= 0. */
SFG_API sfg_status sfg_smooth(sfg_ctx* ctx, const sfg_graph* L, int K, int steps, double omega,
                      uint64_t seed, sfg_dtype storage, void* X_out);
/* Multicolour Gauss-Seidel smoothing, the paper's relaxation (Sec. 3.2: Gauss-Seidel sweeps on
 * L x = 0 from K random vectors orthogonal to the all-one vector). Same seeded block and final
 * projection as sfg_smooth; the sweeps visit the colour classes of a distance-1 colouring
 * (sfg_coloring) in order, each class updated in place and in parallel:
 * x_p <- (1 - omega) x_p + omega (A x)_p / D(p,p) with the current values of all neighbours
 * (omega = 1: plain Gauss-Seidel; 0 < omega < 2). The result equals the sequential sweep over the
 * nodes sorted by (colour, id). The colouring is built on first use and cached with the graph.
 * Layout, storage and errors as sfg_smooth, except omega. */
SFG_API sfg_status sfg_smooth_gs(sfg_ctx* ctx, const sfg_graph* L, int K, int steps, double omega,
                                 uint64_t seed, sfg_dtype storage, void* X_out);

/* Distance-1 colouring used by sfg_smooth_gs (Jones-Plassmann: node priority
 * splitmix64(0x636f6c6f72 xor v), ties by the larger id; each round colours every uncoloured node
 * that outranks its uncoloured neighbours with the smallest colour none of its coloured
 * neighbours holds). color_out (n entries, device, may be NULL) receives colours 0..c-1 and
 * ncolors_host (may be NULL) receives c. Deterministic. Synchronises. */
SFG_API sfg_status sfg_coloring(sfg_ctx* ctx, const sfg_graph* L, int32_t* color_out,
                                int32_t* ncolors_host);

/* Only step 2 of sfg_smooth, in place on a caller-provided block (no init, no projection). */
SFG_API sfg_status sfg_jacobi(sfg_ctx* ctx, const sfg_graph* L, int K, int steps, double omega,
                      sfg_dtype storage, void* X_inout);

/* Tile-shape autotuning of the sweep and the scorer (not in the paper). Variant v of the plain
 * sweep: a warp sweeps TPI = {1, 2, 4, 1, 2, 4}[v] consecutive row tiles before its grid-stride
 * jump, with {4, 4, 4, 3, 3, 3}[v] CTAs per SM requested from the compiler; default v = 1. Shape s
 * of the scorer (sfg_score_edges, sfg_filter_score and the batched forms): a warp scores
 * {1, 2, 1}[s] edge tiles per iteration with {4, 2, 4}[s] CTAs per SM, shape 2 reading rows with
 * loads cached in L2 only; default s = 0 below an average degree of 8, else 1. sfg_autotune times all sweep variants on L (three sweeps each) and both
 * scorer shapes on every edge of L (three launches each), synchronises, and records the fastest of
 * each in ctx's table under (K, storage, degree bucket b: 2^b <= 2m/n < 2^(b+1)); later calls on
 * graphs of that key use them (for the scorer, the key of L_G). Every variant and shape computes
 * the same values bit for bit. sfg_tune_set and sfg_tune_set_score write (or, -1, clear) an entry;
 * sfg_tune_table writes the table as JSON text, one object per key with its sweep variant and
 * scorer shape (-1: none recorded; len_host: its length; SFG_ECAPACITY if cap is too small). */
#define SFG_SWEEP_VARIANTS 6
#define SFG_SCORE_SHAPES 3
SFG_API sfg_status sfg_autotune(sfg_ctx* ctx, const sfg_graph* L, int K, sfg_dtype storage,
                                int* variant_host, double* us_per_sweep_host);
SFG_API sfg_status sfg_tune_set(sfg_ctx* ctx, int K, sfg_dtype storage, int degree_bucket,
                                int variant);
SFG_API sfg_status sfg_tune_set_score(sfg_ctx* ctx, int K, sfg_dtype storage, int degree_bucket,
                                      int shape);
SFG_API sfg_status sfg_tune_table(const sfg_ctx* ctx, char* buf, int64_t cap, int64_t* len_host);

/* ---------------------------------------------------------------------------------------------
 * Spectrally critical edges (Sec. 3.5; scoring and selection steps of Algorithm 1)
 * ------------------------------------------------------------------------------------------- */

/* scores_out[i] = score of canonical edge edge_ids[i] of LG (0 <= id < m), from the two n x K
 * blocks XG (smoothed on L_G) and XP (smoothed on L_P), both in `storage`, per `mode` with
 * eta = 1e-30. FP32 arithmetic. */
SFG_API sfg_status sfg_score_edges(sfg_ctx* ctx, const sfg_graph* LG, const void* XG, const void* XP,
                           int K, sfg_dtype storage, const int32_t* edge_ids, int64_t ne,
                           sfg_score_mode mode, float* scores_out);

/* The filter + score step of edge recovery (Sec. 3.5 with Sec. 3.2's embedding; the embedding and
 * scoring steps of Algorithm 1) in one call: one seeded block (sfg_smooth step 1) is swept `steps` times on L_G
 * and on L_P (same node count), and the listed edges of LG are scored as sfg_score_edges would
 * score the two projected blocks. The projected blocks are not materialised: the projection's
 * mean removal cancels in X_p - X_q and its per-column scaling is applied inside the scorer, so
 * the scores equal sfg_smooth x 2 + sfg_score_edges up to FP32 rounding. Scratch: five n x K
 * blocks. */
SFG_API sfg_status sfg_filter_score(sfg_ctx* ctx, const sfg_graph* LG, const sfg_graph* LP, int K,
                                    int steps, double omega, uint64_t seed, sfg_dtype storage,
                                    const int32_t* edge_ids, int64_t ne, sfg_score_mode mode,
                                    float* scores_out);

/* ids_out[0..k) = the ids of the k largest entries under the strict order (score descending,
 * id ascending), written in ascending id order. ids must be distinct; 0 <= k <= ne else
 * SFG_EINVAL. */
SFG_API sfg_status sfg_select_topk(sfg_ctx* ctx, const float* scores, const int32_t* ids, int64_t ne,
                           int64_t k, int32_t* ids_out);

/* ---------------------------------------------------------------------------------------------
 * Spanning-tree backbone (Sec. 3.1 / 3.4: low-stretch tree approximated by a maximum spanning
 * tree). Maximum-weight spanning forest under the strict order (weight descending, edge id
 * ascending), so the result is unique and equals Kruskal's. Only edges with allow[e] != 0 take
 * part (allow may be NULL). mask_out[e] = 1 for forest edges, else 0. Synchronises.
 * ------------------------------------------------------------------------------------------- */
SFG_API sfg_status sfg_spanning_tree(sfg_ctx* ctx, const sfg_graph* g, const uint8_t* allow,
                             uint8_t* mask_out, int64_t* n_tree_host);

/* ---------------------------------------------------------------------------------------------
 * Spectral coarsening, one level (Sec. 3.2)
 * ------------------------------------------------------------------------------------------- */

/* delta_out[e] = 1 - (X_p . X_q)^2 / (||X_p||^2 ||X_q||^2) for every canonical edge e = (p, q)
 * (the algebraic-distance affinity quoted in Sec. 3.2), evaluated in FP64 without fused
 * multiply-add, in increasing k order, from the FP32 block X (n x K). A zero row gives 1. */
SFG_API sfg_status sfg_affinity(sfg_ctx* ctx, const sfg_graph* L, const float* X, int K,
                        double* delta_out);

/* Allocation-free sfg_affinity. The paper has no counterpart: this entry point exists for callers
 * that cannot let a library allocate device memory (applications that give all device memory to
 * their own pool, runtimes that must keep the device footprint fixed after start-up, code running
 * where cudaMalloc / cudaMallocAsync are not permitted). Same arguments and the same bit-exact
 * result as sfg_affinity, but its scratch (one FP64 row norm per node) is a fixed file-scope
 * device array of SFG_AFFINITY_NOALLOC_MAX_N entries (8 MiB); the call itself allocates nothing.
 *  - The array is taken once per device, when the first context on that device is created:
 *    sfg_ctx_create looks up its device address (cudaGetSymbolAddress, with that device current),
 *    which loads the module that holds it. From then on the device keeps the 8 MiB until the
 *    process exits, and no sfg_affinity_noalloc call takes any memory.
 *  - n > SFG_AFFINITY_NOALLOC_MAX_N gives SFG_ECAPACITY (use sfg_affinity).
 *  - Every call on a device shares the one array: calls whose work overlaps on the GPU (several
 *    streams or contexts at once) race on it. Serialise them, e.g. on one stream. */
#define SFG_AFFINITY_NOALLOC_MAX_N (1 << 20)
SFG_API sfg_status sfg_affinity_noalloc(sfg_ctx* ctx, const sfg_graph* L, const float* X, int K,
                                        double* delta_out);

/* One coarsening level from a block X (n x K, row-major, `storage` SFG_F32 or SFG_BF16; entries
 * widened exactly to FP64): affinities as sfg_affinity; each node hooks to the neighbour with the
 * smallest delta (ties: smaller id); aggregation sets S_i are the connected components of the
 * hooks, numbered by increasing smallest member (agg_out[p] = i for p in S_i); the coarse
 * Laplacian is the Galerkin product H^-T L H^+ of Sec. 3.2, i.e. the canonical form of the list
 * (agg[u], agg[v], w) taken in fine edge-id order. fine2coarse_out[e] (may be NULL) = coarse edge
 * id of fine edge e, or -1 inside an aggregate. Synchronises. */
SFG_API sfg_status sfg_coarsen(sfg_ctx* ctx, const sfg_graph* L, const void* X, int K,
                               sfg_dtype storage, int32_t* agg_out, int32_t* fine2coarse_out,
                               int32_t* n_coarse_host, sfg_graph** coarse_out);

/* Backward mapping of Sec. 3.4 (the backward-mapping step of Algorithm 1): pmask_f[e] over the fine graph's edges =
 * union of a maximum spanning tree of each aggregation set's induced subgraph, and, for every
 * coarse edge (I, J) with pmask_c set, the heaviest fine edge between S_I and S_J (ties: smallest
 * id). agg and fine2coarse as produced by sfg_coarsen. Synchronises. */
SFG_API sfg_status sfg_backward_map(sfg_ctx* ctx, const sfg_graph* fine, const int32_t* agg,
                            const int32_t* fine2coarse, const sfg_graph* coarse,
                            const uint8_t* pmask_c, uint8_t* pmask_f);

/* ---------------------------------------------------------------------------------------------
 * The method (Algorithm 1)
 * ------------------------------------------------------------------------------------------- */
typedef struct {
    int K;              /* vectors per block */
    int steps;          /* Jacobi sweeps per embedding */
    int levels;         /* 0: flat (spanning tree + recovered edges); >= 1: coarsening levels */
    double omega;       /* Jacobi weight, e.g. 0.7 */
    uint64_t seed;      /* level l embeds with seed (l = 0) or splitmix64(seed ^ l) */
    sfg_score_mode mode;
    double budget_frac; /* beta: each level ends with round(beta * base) edges beyond a forest */
    int budget_unit;    /* 0: base = N_l; 1: base = number of off-tree edges of G_l */
    sfg_dtype storage;  /* vector block storage */
    int smoother;       /* SFG_SMOOTH_JACOBI (omega in (0, 1]) or SFG_SMOOTH_GAUSS_SEIDEL
                           (multicolour, sfg_smooth_gs; omega in (0, 2), 1 = plain) */
} sfg_params;

/* Smoothers of sfg_params.smoother. */
enum { SFG_SMOOTH_JACOBI = 0, SFG_SMOOTH_GAUSS_SEIDEL = 1 };

/* The method (Algorithm 1 of Sec. 3.6: graph in; sparsifier and coarsening hierarchy out).
 * mask_out[e] (m entries) = 1 for the edges of the sparsifier P of G. Flat: maximum spanning
 * forest, then the top-scored off-tree edges. Multilevel: coarsen `levels` times (the
 * aggregation always from FP32 embeddings, so params->storage changes only the edge-recovery
 * blocks; stopping early if a level has no edges left), sparsify the
 * coarsest graph flat, then at each finer level map the sparsifier back (sfg_backward_map),
 * re-embed, score the edges outside it and add the top ones. Budget at each level: the level's
 * sparsifier gets round-half-up(beta * base) edges beyond N_l - c_l (c_l = number of components),
 * counting edges already mapped; none are added if it is already over. n_selected_host (may be
 * NULL) receives the number of edges in P. hier_out (may be NULL) receives the hierarchy: the
 * graphs G_1 .. G_lf, the maps H_1 .. H_lf and every level's sparsifier P_0 .. P_lf (a flat run
 * has lf = 0), to be released with sfg_hierarchy_destroy. Synchronises. */
SFG_API sfg_status sfg_sparsify(sfg_ctx* ctx, const sfg_graph* G, const sfg_params* params,
                                uint8_t* mask_out, int64_t* n_selected_host,
                                sfg_hierarchy** hier_out);

/* Accessors of a hierarchy (Algorithm 1's [G_1 .. G_lf; H_1 .. H_lf] plus the sparsifier P_l of
 * every level). Level 0 is the input graph G (borrowed: it must outlive the hierarchy), levels
 * 1 .. lf are the coarse graphs, owned by the hierarchy (do not destroy them).
 * sfg_hierarchy_levels: lf. sfg_hierarchy_graph: G_level. sfg_hierarchy_map (level 1 .. lf): the
 * map H_level from G_{level-1} to G_level as agg_out (N_{level-1} entries, node -> aggregate) and
 * fine2coarse_out (M_{level-1} entries, edge -> coarse edge or -1), each may be NULL, as
 * sfg_coarsen writes them. sfg_hierarchy_mask (level 0 .. lf): P_level over G_level's canonical
 * edges (M_level entries; level 0 equals sfg_sparsify's mask_out). Out-of-range levels give
 * SFG_EINVAL. The copies are stream-ordered on ctx's stream. */
SFG_API sfg_status sfg_hierarchy_levels(const sfg_hierarchy* h, int* levels_host);
SFG_API sfg_status sfg_hierarchy_graph(const sfg_hierarchy* h, int level, const sfg_graph** out);
SFG_API sfg_status sfg_hierarchy_map(sfg_ctx* ctx, const sfg_hierarchy* h, int level,
                                     int32_t* agg_out, int32_t* fine2coarse_out);
SFG_API sfg_status sfg_hierarchy_mask(sfg_ctx* ctx, const sfg_hierarchy* h, int level,
                                      uint8_t* mask_out);
SFG_API void sfg_hierarchy_destroy(sfg_hierarchy* h);

/* Batched flat method: sparsify ng independent graphs in one set of launches (their disjoint
 * union is processed as one graph; the seeded blocks, projection statistics, budgets and top-k
 * are per graph). masks_out[g] is a device buffer of graph g's m_g entries; n_selected_host (may
 * be NULL) receives ng counts. Each graph's mask is the one sfg_sparsify gives for that graph
 * with the same parameters (up to FP32 summation order in the column statistics). levels must be
 * 0 (else SFG_EUNSUPPORTED); the union must fit int32 indices (sum n < 2^31, 2 sum m < 2^31).
 * Synchronises. */
SFG_API sfg_status sfg_sparsify_batched(sfg_ctx* ctx, int ng, const sfg_graph* const* gs,
                                        const sfg_params* params, uint8_t* const* masks_out,
                                        int64_t* n_selected_host);

/* Batch plan: the same batched flat method split into a plan, built once per set of graphs, and
 * runs of it. sfg_batch_create (synchronises) joins the graphs, computes every graph's spanning
 * forest, candidate edges and budget (params as sfg_sparsify_batched; params->seed is not used).
 * flags (bits; any other bit is SFG_EINVAL):
 *  - SFG_BATCH_AUTOTUNE: time the sweep's tile shapes and the scorer's launch shapes on the union
 *    of the graphs and on the union of their forests and record the fastest in ctx's table
 *    (sfg_autotune);
 *  - SFG_BATCH_LOCALITY: renumber each graph's nodes internally by breadth-first level from a
 *    pseudo-peripheral root (not in the paper; a memory-locality device for graphs whose input
 *    order scatters neighbours, e.g. k-NN graphs of unsorted points; at most 4096 levels, nodes
 *    further out and other components keep their input order after the labelled ones). Seeded rows are drawn from
 *    the original node ids, forest ties and the selection use the original edge ids, and masks
 *    come out in the original edge order, so the result is the plan's without the flag up to FP32
 *    summation order in the sweeps and column statistics.
 * sfg_batch_run
 * writes the sparsifiers of all graphs for one seed into mask_out (a device buffer of
 * edges_host entries: graph g's m_g edges at [edge_offsets_host[g], edge_offsets_host[g + 1]),
 * in its canonical order); it only queues kernels and stream-ordered allocations on ctx's stream
 * (no host synchronisation), so it can be captured in a CUDA graph and replayed, and every run
 * with the same seed gives the same bits. sfg_batch_info gives the number of graphs, the total
 * edge count, the ng + 1 edge offsets and every graph's sparsifier size (each pointer may be
 * NULL). The plan holds its own copy of the graphs: they may be destroyed after
 * sfg_batch_create. */
typedef struct sfg_batch sfg_batch;
#define SFG_BATCH_AUTOTUNE 1
#define SFG_BATCH_LOCALITY 2
SFG_API sfg_status sfg_batch_create(sfg_ctx* ctx, int ng, const sfg_graph* const* gs,
                                    const sfg_params* params, int flags, sfg_batch** out);
SFG_API sfg_status sfg_batch_info(const sfg_batch* b, int* ng_host, int64_t* edges_host,
                                  int64_t* edge_offsets_host, int64_t* n_selected_host);
SFG_API sfg_status sfg_batch_run(sfg_ctx* ctx, const sfg_batch* b, uint64_t seed,
                                 uint8_t* mask_out);
SFG_API void sfg_batch_destroy(sfg_batch* b);

/* Relative condition number kappa(L_G, L_P) of Sec. 2.2 (Eq. eqn:ineq), the paper's measure of
 * sparsifier quality, for P = the edges of G with mask[e] != 0 (m entries, device). kappa =
 * lambda_max / lambda_min of L_G x = lambda L_P x on the complement of the common null space,
 * estimated from `steps` steps of FP64 Lanczos on L_P^+ L_G in the L_P inner product with full
 * reorthogonalisation, started from a vector seeded by `seed`; the Krylov dimension is capped at
 * n - (number of components), at which the Ritz values are the exact eigenvalues up to FP64
 * rounding. Each L_P solve eliminates degree <= 2 nodes exactly (parallel rounds) and solves the
 * remaining core by preconditioned CG to a relative residual of 1e-13 of its own right-hand side
 * or 1e-12 of the whole one (not in the paper: its experiments report kappa but not how it is
 * computed). The iteration stops early when the Krylov space is exhausted (beta below 1e-10 of
 * the largest alpha, a vanishing residual, or a core solve that fails once at least half of the
 * Krylov dimension has been explored, which happens on a right-hand side made of rounding noise).
 * kappa_host receives kappa (+infinity
 * if P does not span every component of G; 1 if G has no edges). lambda_min is exactly 1 when
 * G \ P has more components than G (L_G >= L_P, with equality on the vectors that are constant on
 * the components of G \ P); that case is detected and used instead of the Ritz value. info_host
 * (may be NULL, 6 entries) receives {lambda_min, lambda_max, Lanczos steps taken, core CG
 * iterations in all, 1 if the last step ended on a failed core solve else 0, 1 if lambda_min = 1
 * was certified by the component count else 0}. Deterministic. Errors: SFG_EINVAL
 * (bad arguments), SFG_ENOMEM (it keeps 2 (steps + 1) FP64 vectors of n entries), SFG_ETIMEOUT
 * (the core CG did not converge before half of the Krylov dimension: a core too ill-conditioned
 * for CG at the tolerance; no kappa is returned then). Synchronises. */
SFG_API sfg_status sfg_kappa(sfg_ctx* ctx, const sfg_graph* G, const uint8_t* mask, int steps,
                             uint64_t seed, double* kappa_host, double* info_host);

/* Sparsification to a target condition number: P is sigma-similar to G when kappa(L_G, L_P) <=
 * sigma^2 (Sec. 2.2, Eq. eqn:ineq); Sec. 3.4 builds sparsifiers for a desired kappa and
 * Algorithm 1 takes sigma as its argument. Flat form: P starts as the maximum spanning forest of G;
 * each round r = 0, 1, ... measures kappa(L_G, L_P) with sfg_kappa (kappa_steps Lanczos steps) and
 * stops once it is <= kappa_target (= sigma^2) or r = max_rounds; otherwise it re-embeds G and the
 * current P from params->seed (params->K, steps, omega, storage, mode), scores every edge of G
 * outside P and adds the top ones, so that after round r + 1 P holds round-half-up((r + 1) *
 * batch_frac * base) edges beyond the forest (base = n or the number of off-forest edges, per
 * params->budget_unit; params->budget_frac is not used). Stops early when no edge is left to add.
 * mask_out (m entries) receives P; n_selected_host, kappa_trace_host (max_rounds + 1 entries:
 * kappa after each round, the last entry written is the final kappa) and rounds_host (rounds of
 * additions performed) may be NULL. params->levels must be 0 (else SFG_EINVAL); kappa_target >= 1,
 * batch_frac > 0, max_rounds >= 0, kappa_steps >= 1. Synchronises. */
SFG_API sfg_status sfg_sparsify_to_kappa(sfg_ctx* ctx, const sfg_graph* G, const sfg_params* params,
                                         double kappa_target, double batch_frac, int max_rounds,
                                         int kappa_steps, uint8_t* mask_out,
                                         int64_t* n_selected_host, double* kappa_trace_host,
                                         int* rounds_host);

/* Solve L_G x = b by conjugate gradients preconditioned with the sparsifier P = the edges of G
 * with mask[e] != 0 (the use the paper makes of its sparsifiers in its PCG experiments, Table 3):
 * each iteration applies L_P^+ exactly (the elimination solver of sfg_kappa: degree <= 2 nodes
 * eliminated in rounds, the core by CG to 1e-13). mask == NULL selects the diagonal (Jacobi)
 * preconditioner instead, as a baseline. b (n entries, FP64, device, read only) is first
 * projected onto the range of L_G (its mean removed on every connected component); x (n entries,
 * FP64, device) receives the solution with mean zero on every component. Stops when
 * ||r||_2 <= tol ||b_projected||_2 or after maxit iterations; iters_host and relres_host (may be
 * NULL) receive the iterations taken and the final relative residual (recursive). All sums run
 * in a fixed order: deterministic. Errors: SFG_EINVAL (bad arguments, or P does not span the
 * components of G), SFG_ENOMEM, SFG_ETIMEOUT (a core solve did not converge). Synchronises. */
SFG_API sfg_status sfg_solve_pcg(sfg_ctx* ctx, const sfg_graph* G, const uint8_t* mask,
                                 const double* b, double tol, int maxit, double* x, int* iters_host,
                                 double* relres_host);

/* ---------------------------------------------------------------------------------------------
 * Learned edge proposals (an addition to the paper's method; the paper has no learned part).
 * A small network predicts each candidate edge's score after `steps` sweeps from features of a
 * much shorter embedding; its best guesses are rescored by the plain method, which therefore
 * stays both the fallback and the final arbiter of selection.
 * Features (16 per edge, FP32, row-major), for e = (p, q) with weighted degree d, neighbour count
 * deg and the projected-embedding distances s_G, s_P of sfg_score_edges (modes G and P) after
 * `steps` sweeps from `seed`: ln w, ln d_p + ln d_q, |ln d_p - ln d_q|, ln(s_G + 1e-30),
 * ln(s_P + 1e-30), ln(s_P + 1e-30) - ln(s_G + 1e-30), ln(deg_p deg_q), ln(s_G + s_P + 1e-30), 0 x 8.
 * Network: 16 -> 64 -> 64 -> 1 with ReLU, BF16 operands on tensor cores, FP32 accumulation and
 * FP32 master parameters, flat in the order W1 [16][64] (in x out), b1 [64], W2 [64][64], b2,
 * w3 [64], b3: SFG_MLP_NPARAM values. Loss: mean squared error. Training: Adam (beta 0.9,
 * 0.999, eps 1e-8) over consecutive minibatches; gradients are deterministic.
 * Initial weights: Kaiming-uniform, weight j = (2u - 1) sqrt(6 / fan_in) with
 * u = (splitmix64(splitmix64(seed) + j * 0x9E3779B97F4A7C15) >> 11) 2^-53; biases 0.
 * ------------------------------------------------------------------------------------------- */
#define SFG_MLP_NPARAM 5313
#define SFG_MLP_NFEAT 16
typedef struct sfg_mlp sfg_mlp;
SFG_API sfg_status sfg_mlp_create(sfg_ctx* ctx, uint64_t seed, sfg_mlp** out);
SFG_API void sfg_mlp_destroy(sfg_mlp* net);
/* Copy the FP32 parameters out / in (set also clears the Adam state). */
SFG_API sfg_status sfg_mlp_params(sfg_ctx* ctx, const sfg_mlp* net, float* theta_out);
SFG_API sfg_status sfg_mlp_set_params(sfg_ctx* ctx, sfg_mlp* net, const float* theta);
/* out[i] = network output for feature row i (ne rows), on the tcgen05 tensor cores. Queued
 * without synchronisation (it can be captured in a CUDA graph); every completion wait inside the
 * kernel is bounded by a clock, and a wait that runs out is reported by the next sfg_mlp_check
 * (or by a synchronising call of the network: sfg_mlp_gradient / sfg_mlp_train with loss_host,
 * sfg_sparsify_learned) as SFG_ETIMEOUT. */
SFG_API sfg_status sfg_mlp_forward(sfg_ctx* ctx, const sfg_mlp* net, const float* feats,
                                   int64_t ne, float* out);
/* Synchronise ctx's stream; SFG_ETIMEOUT (once) if a bounded completion wait of this network's
 * tensor-core kernels ran out since the last check, else SFG_OK. */
SFG_API sfg_status sfg_mlp_check(sfg_ctx* ctx, const sfg_mlp* net);
/* Gradient of mean((y - targets)^2) over the ne rows (grad_out: SFG_MLP_NPARAM FP32, may be
 * NULL); loss_host (may be NULL) receives the loss and synchronises. Forward and backward run on
 * the tcgen05 tensor cores, 128 rows per tile: BF16 operands (features, W1, W2, the first hidden
 * layer and the two backward deltas), FP32 accumulation in TMEM; the weight gradients contract
 * over each tile's rows and accumulate in TMEM across the tiles of a CTA, the CTAs' partial
 * gradients are added in a fixed order (deterministic). */
SFG_API sfg_status sfg_mlp_gradient(sfg_ctx* ctx, sfg_mlp* net, const float* feats,
                                    const float* targets, int64_t ne, float* grad_out,
                                    double* loss_host);
/* `epochs` passes of Adam steps over consecutive minibatches of `batch` rows; loss_host (may be
 * NULL) receives the final full-data loss and synchronises. */
SFG_API sfg_status sfg_mlp_train(sfg_ctx* ctx, sfg_mlp* net, const float* feats,
                                 const float* targets, int64_t ne, int64_t batch, int epochs,
                                 double lr, double* loss_host);
/* Feature rows (ne x 16) of the listed edges of LG (see above); LP: the current sparsifier. */
SFG_API sfg_status sfg_edge_features(sfg_ctx* ctx, const sfg_graph* LG, const sfg_graph* LP, int K,
                                     int steps, double omega, uint64_t seed, sfg_dtype storage,
                                     const int32_t* edge_ids, int64_t ne, float* feats_out);
/* Flat method with learned proposals: spanning forest; features of every off-tree edge from a
 * feat_steps embedding; the network's top round(propose_frac * candidates) edges (at least the
 * budget k) are rescored by sfg_filter_score with params->steps and the top k of them are added.
 * net == NULL or propose_frac >= 1 gives the plain flat method. params->levels must be 0. */
SFG_API sfg_status sfg_sparsify_learned(sfg_ctx* ctx, const sfg_graph* G, const sfg_params* params,
                                        const sfg_mlp* net, int feat_steps, double propose_frac,
                                        uint8_t* mask_out, int64_t* n_selected_host);

#ifdef __cplusplus
}
#endif
#endif /* SFG_H */
