// Internal declarations shared by the translation units of libsfg (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <algorithm>
#include <map>
#include <cstdio>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/sfg.h"

// ------------------------------------------------------------------------------------------------
// Context: device, borrowed stream, last error text, optional per-kernel event timers.
// ------------------------------------------------------------------------------------------------
struct sfg_timer_rec {
    const char* name;
    cudaEvent_t start, stop;
};

struct sfg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;          // the device's stream-ordered pool of the library
    int* host_word = nullptr;              // pinned host ints for flags read after a sync
    int num_sms = 0;
    std::string last_error;
    bool timing = false;
    std::vector<sfg_timer_rec> timers;     // recorded this session
    std::vector<cudaEvent_t> event_pool;   // free events
    int64_t launches = 0;                  // kernels launched through this context
    std::map<uint32_t, int> tune;          // (K, dtype, degree bucket) -> sweep variant
    std::map<uint32_t, int> score_tune;    // (K, dtype, degree bucket) -> scorer launch shape
    std::map<std::tuple<const void*, int, size_t>, int> occupancy;  // resident CTAs per SM
    int64_t alloc_count = 0;               // for the allocation-failure injection hook
    int64_t fail_alloc_at = -1;            // SFG_FAULT_ALLOC=<n>: the n-th allocation fails
    bool withhold_mma = false;             // SFG_FAULT_MMA_WAIT=1: tensor-core kernels issue no
                                           // MMA, so their bounded completion waits run out
};

struct sfg_graph {
    int device = -1;           // device that holds the arrays
    int32_t n = 0;
    int64_t m = 0;             // canonical edges
    int32_t* eu = nullptr;     // [m] canonical edge endpoints, eu < ev, sorted
    int32_t* ev = nullptr;
    float* ew = nullptr;       // [m]
    int32_t* row_ptr = nullptr;// [n+1]
    int2* colval = nullptr;    // [2m] (column, float bits of the weight), rows sorted by column
    int32_t* eid = nullptr;    // [2m] canonical edge id of each CSR entry
    double* deg = nullptr;     // [n]
    double* invdeg = nullptr;  // [n] 1 / deg in FP64 (0 for isolated nodes)
    // Gauss-Seidel colouring, built on first use (color.cu): colour per node, the nodes sorted
    // by (colour, id), and colour c's nodes at gs_order[gs_off[c], gs_off[c + 1]).
    int32_t* gs_color = nullptr;
    int32_t* gs_order = nullptr;
    std::vector<int64_t> gs_off;
    // Rows with more entries than the sweep's heavy-row threshold, built on the first sweep
    // (smooth.cu): hv_n rows (-1 = not built yet) at hv_rows, row h's segments at
    // hv_seg[hv_soff[h], hv_soff[h + 1]), each (row, first entry, end entry, 0).
    int32_t hv_n = -1;
    int64_t hv_nseg = 0;
    int32_t* hv_rows = nullptr;
    int32_t* hv_soff = nullptr;
    int4* hv_seg = nullptr;
    // The same rows grouped by Gauss-Seidel colour class (built on the first Gauss-Seidel
    // smoothing): gh_rows sorted by (colour, id), row k's segments at gh_seg[gh_soff[k],
    // gh_soff[k + 1]); colour c's rows at [gh_coff[c], gh_coff[c + 1]) and its segments at
    // [gh_scoff[c], gh_scoff[c + 1]).
    bool gh_ready = false;
    int32_t* gh_rows = nullptr;
    int32_t* gh_soff = nullptr;
    int4* gh_seg = nullptr;
    std::vector<int64_t> gh_coff, gh_scoff;
    cudaStream_t stream = nullptr;
};

// Every entry point runs with the context's device current and gives the caller's current device
// back when it returns (cudaSetDevice only when the two differ).
struct SfgDeviceGuard {
    int prev = -1;
    explicit SfgDeviceGuard(int device) {
        int cur = -1;
        if (device < 0 || cudaGetDevice(&cur) != cudaSuccess || cur == device) return;
        if (cudaSetDevice(device) == cudaSuccess) prev = cur;
        else cudaGetLastError();  // the entry point's own CUDA calls then report the failure
    }
    ~SfgDeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    SfgDeviceGuard(const SfgDeviceGuard&) = delete;
    SfgDeviceGuard& operator=(const SfgDeviceGuard&) = delete;
};
#define SFG_DEVICE(ctx) SfgDeviceGuard sfg_device_guard_((ctx)->device)

// ------------------------------------------------------------------------------------------------
// Status helpers. Every API entry point returns through these so the text lands in ctx.
// ------------------------------------------------------------------------------------------------
sfg_status sfg_fail(sfg_ctx* ctx, sfg_status st, const char* fmt, ...);
sfg_status sfg_cuda_fail(sfg_ctx* ctx, cudaError_t e, const char* where);

#define SFG_CUDA(ctx, call)                                                 \
    do {                                                                    \
        cudaError_t _e = (call);                                            \
        if (_e != cudaSuccess) return sfg_cuda_fail((ctx), _e, #call);      \
    } while (0)

#define SFG_TRY(call)                                                       \
    do {                                                                    \
        sfg_status _s = (call);                                             \
        if (_s != SFG_OK) return _s;                                        \
    } while (0)

#define SFG_LAUNCH_CHECK(ctx, name)                                         \
    do {                                                                    \
        cudaError_t _e = cudaGetLastError();                                \
        if (_e != cudaSuccess) return sfg_cuda_fail((ctx), _e, name);       \
    } while (0)

// Stream-ordered device allocation from the context's pool (cudaMallocAsync).
sfg_status sfg_alloc(sfg_ctx* ctx, void** p, size_t bytes);
void sfg_free(sfg_ctx* ctx, void* p);

// Scoped list of scratch allocations released (stream-ordered) at scope exit.
struct Scratch {
    sfg_ctx* ctx;
    std::vector<void*> ptrs;
    explicit Scratch(sfg_ctx* c) : ctx(c) {}
    ~Scratch() {
        for (void* p : ptrs) sfg_free(ctx, p);
    }
    template <typename T>
    sfg_status get(T** p, size_t count) {
        void* q = nullptr;
        sfg_status s = sfg_alloc(ctx, &q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
        if (s != SFG_OK) return s;
        ptrs.push_back(q);
        *p = static_cast<T*>(q);
        return SFG_OK;
    }
    void release(void* p) {  // hand ownership to the caller
        for (auto& q : ptrs)
            if (q == p) q = nullptr;
    }
};

// The context's pinned host ints (allocated on first use): a stream-ordered copy into one costs no
// synchronisation, and the host reads it after the next one. Slots: 0 spanning-forest round
// flag, 1 pointer-jumping flag.
constexpr int kSfgHostWords = 4;
sfg_status sfg_host_word(sfg_ctx* ctx, int slot, int** out);

// Kernel timing (no-ops unless ctx->timing).
void sfg_tic(sfg_ctx* ctx, const char* name);
void sfg_toc(sfg_ctx* ctx);

// Pointer checks: NULL or not device-accessible memory -> SFG_EINVAL.
sfg_status sfg_check_dev(sfg_ctx* ctx, const void* p, const char* what);

// Grid size for a grid-stride kernel: a whole number of waves over the SMs.
int sfg_grid(sfg_ctx* ctx, const void* kernel, int block, size_t smem, int64_t work_items);

static inline unsigned ceil_div_u(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------------------------------------------
// Device primitives (primitives.cu)
// ------------------------------------------------------------------------------------------------
// out[i] = sum_{j<i} in[j] for i in [0, n]; out has n + 1 entries (out[n] = total).
sfg_status sfg_scan_u8(sfg_ctx* ctx, const uint8_t* in, int64_t* out, int64_t n);
sfg_status sfg_scan_i32(sfg_ctx* ctx, const int32_t* in, int64_t* out, int64_t n);
sfg_status sfg_scan_i64(sfg_ctx* ctx, const int64_t* in, int64_t* out, int64_t n);
// Stable LSD radix sort of (key, val) pairs on the low `bits` bits of the keys. The sorted data
// ends in (*keys, *vals); the pointers may be swapped with the alternate buffers.
sfg_status sfg_radix_sort_pairs(sfg_ctx* ctx, uint64_t** keys, uint32_t** vals,
                                uint64_t** keys_alt, uint32_t** vals_alt, int64_t n, int bits);
// Copy scalars back (synchronises the stream).
sfg_status sfg_read_i64(sfg_ctx* ctx, const int64_t* dev, int64_t* host);

// ------------------------------------------------------------------------------------------------
// Cross-unit helpers
// ------------------------------------------------------------------------------------------------
// Build an sfg_graph from an input edge list already on the device (validated or not).
sfg_status sfg_build_graph(sfg_ctx* ctx, int32_t n, int64_t m, const int32_t* u,
                           const int32_t* v, const float* w, bool validate, sfg_graph** out,
                           int32_t* fine2coarse_out);
sfg_status sfg_subgraph_impl(sfg_ctx* ctx, const sfg_graph* g, const uint8_t* mask,
                             sfg_graph** out);
// comp_out (optional, n entries): each node's component label, a node of that component.
// key_id (m entries, may be NULL): the id that breaks weight ties for edge e (default e), with
// key_inv its inverse; a relabelled copy of a graph passes its original edge ids, so that its
// forest is the original graph's forest edge for edge.
sfg_status sfg_mst_impl(sfg_ctx* ctx, const sfg_graph* g, const uint8_t* allow, uint8_t* mask,
                        int64_t* n_tree, int32_t* comp_out = nullptr,
                        const int32_t* key_id = nullptr, const int32_t* key_inv = nullptr);
sfg_status sfg_smooth_impl(sfg_ctx* ctx, const sfg_graph* L, int K, int steps, double omega,
                           uint64_t seed, sfg_dtype storage, void* X_out);
// sg, sp (may be NULL): per-column scales applied to raw blocks (projection folded in).
sfg_status sfg_score_impl(sfg_ctx* ctx, const sfg_graph* LG, const void* XG, const void* XP,
                          int K, sfg_dtype storage, const int32_t* ids, int64_t ne,
                          sfg_score_mode mode, float* out, const float* sg = nullptr,
                          const float* sp = nullptr);
sfg_status sfg_score_batched_impl(sfg_ctx* ctx, const sfg_graph* LG, const void* XG,
                                  const void* XP, int K, sfg_dtype storage, const int32_t* ids,
                                  int64_t ne, sfg_score_mode mode, float* out, const float* sg,
                                  const float* sp, const int32_t* node_off, int ngraphs);
// orig_local (n entries, may be NULL): the graph-local node id whose seeded row row r carries
// (default r - node_off[g]), for unions whose nodes were reordered.
sfg_status sfg_filter_score_batched_impl(sfg_ctx* ctx, const sfg_graph* U, const sfg_graph* PU,
                                         const int32_t* orig_local,
                                         int ng, const int32_t* node_off, int K, int steps,
                                         double omega, uint64_t seed, sfg_dtype storage,
                                         const int32_t* ids, int64_t ne, sfg_score_mode mode,
                                         float* scores);
// Top-k per segment: candidates [seg_off[s], seg_off[s+1]) of segment s keep their k_dev[s]
// largest; the chosen ids of all segments are written in ascending order (out has sum k entries).
sfg_status sfg_topk_segmented_impl(sfg_ctx* ctx, const float* scores, const int32_t* ids,
                                   int64_t ne, int nseg, const int64_t* seg_off,
                                   const int64_t* k_dev, int64_t k_total, int32_t* out);
typedef struct sfg_mlp sfg_mlp;
sfg_status sfg_mlp_forward_impl(sfg_ctx* ctx, const sfg_mlp* net, const float* feats, int64_t ne,
                                float* out);
sfg_status sfg_mlp_check_impl(sfg_ctx* ctx, const sfg_mlp* net);
sfg_status sfg_edge_features_impl(sfg_ctx* ctx, const sfg_graph* LG, const sfg_graph* LP, int K,
                                  int steps, double omega, uint64_t seed, sfg_dtype storage,
                                  const int32_t* ids, int64_t ne, float* feats);
sfg_status sfg_filter_score_impl(sfg_ctx* ctx, const sfg_graph* LG, const sfg_graph* LP, int K,
                                 int steps, double omega, uint64_t seed, sfg_dtype storage,
                                 const int32_t* ids, int64_t ne, sfg_score_mode mode,
                                 float* scores);
sfg_status sfg_topk_impl(sfg_ctx* ctx, const float* scores, const int32_t* ids, int64_t ne,
                         int64_t k, int32_t* out);
sfg_status sfg_coarsen_impl(sfg_ctx* ctx, const sfg_graph* L, const void* X, int K,
                            sfg_dtype storage, int32_t* agg, int32_t* f2c, int32_t* nc,
                            sfg_graph** coarse);
sfg_status sfg_backward_impl(sfg_ctx* ctx, const sfg_graph* fine, const int32_t* agg,
                             const int32_t* f2c, const sfg_graph* coarse, const uint8_t* pmask_c,
                             uint8_t* pmask_f);
void sfg_graph_free(sfg_graph* g);
// Device arrays of a graph with n nodes and m canonical edges (contents unset).
sfg_status sfg_alloc_graph(sfg_ctx* ctx, int32_t n, int64_t m, sfg_graph** out);
bool sfg_k_supported(int K, sfg_dtype dt);
// Tile-shape tuning table of a context (see sfg_autotune). Variant -1 = none recorded.
int sfg_degree_bucket(const sfg_graph* L);
uint32_t sfg_tune_key(int K, sfg_dtype dt, int bucket);
int sfg_tuned_variant(const sfg_ctx* ctx, int K, sfg_dtype dt, const sfg_graph* L);
void sfg_tune_record(sfg_ctx* ctx, int K, sfg_dtype dt, const sfg_graph* L, int variant);
// Launch shape of the scorer for graphs like L: the recorded one, else 0 (one tile per warp
// iteration, four CTAs per SM) below an average degree of 8 and 1 (two tiles, two CTAs) above.
int sfg_score_shape(const sfg_ctx* ctx, int K, sfg_dtype dt, const sfg_graph* L);
// Times both scorer shapes on every edge of L with X as both blocks and records the faster.
sfg_status sfg_score_autotune_impl(sfg_ctx* ctx, const sfg_graph* L, int K, sfg_dtype storage,
                                   const void* X);
sfg_status sfg_autotune_impl(sfg_ctx* ctx, const sfg_graph* L, int K, sfg_dtype storage,
                             int* best, double* us);

// splitmix64 (Steele, Lea & Flood 2014), host and device.
__host__ __device__ inline uint64_t sfg_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// kappa(L_G, L_P) for P = the masked edges of G (kappa.cu); info6 (nullable) as sfg_kappa's.
sfg_status sfg_kappa_impl(sfg_ctx* ctx, const sfg_graph* G, const uint8_t* mask, int steps,
                          uint64_t seed, double* kappa, double* info6);
// Build the Gauss-Seidel colouring of L once (cached on the graph; color.cu).
sfg_status sfg_gs_prepare(sfg_ctx* ctx, const sfg_graph* L);
// Rows with more than SFG_HEAVY_ROW entries and their SFG_HEAVY_SEG-entry segments (hv_* of the
// graph), built once per graph (smooth.cu); the sweep and the spanning-forest rounds use them.
constexpr int32_t SFG_HEAVY_ROW = 256, SFG_HEAVY_SEG = 128;
sfg_status sfg_heavy_prepare(sfg_ctx* ctx, const sfg_graph* L);
// Give P (a subgraph of G on the same nodes) G's colouring, which is proper for P too.
sfg_status sfg_gs_inherit(sfg_ctx* ctx, const sfg_graph* P, const sfg_graph* G);
// y_p = d_p - omega * (weight to nodes after p in (colour, id) order): the weights of the
// quantity y^T x that the colour-ordered SOR sweep conserves (color.cu).
__global__ void k_gs_weights(int32_t n, const int32_t* __restrict__ row_ptr,
                             const int2* __restrict__ colval, const int32_t* __restrict__ color,
                             double omega, double* __restrict__ y);
__global__ void k_gs_weights_heavy(int32_t nh, const int32_t* __restrict__ hrow,
                                   const int32_t* __restrict__ row_ptr, const int2* __restrict__ colval,
                                   const int32_t* __restrict__ color, double omega, double* __restrict__ y);
sfg_status sfg_smooth_gs_impl(sfg_ctx* ctx, const sfg_graph* L, int K, int steps, double omega,
                              uint64_t seed, sfg_dtype storage, void* X_out);
sfg_status sfg_pointer_jump(sfg_ctx* ctx, int32_t n, const int32_t* comp, int32_t* parent);
sfg_status sfg_count_mask(sfg_ctx* ctx, const uint8_t* mask, int64_t m, int64_t* count_host);
sfg_status sfg_affinity_impl(sfg_ctx* ctx, const sfg_graph* L, const void* X, int K,
                             sfg_dtype storage, double* delta);
// Resolve (once per device, with ctx's device current) the device address of the file-scope
// scratch of the allocation-free entry points (noalloc.cu); called by sfg_ctx_create.
sfg_status sfg_noalloc_prepare(sfg_ctx* ctx);
