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
// Rows with more than 256 entries (the hubs of power-law graphs) would hold one lane group, and
// with it its warp, for the whole sweep; they are swept apart in fixed 128-entry segments whose
// partial sums are added in order (k_heavy_part, k_heavy_final), so results stay deterministic.
//
// The first sweep also removes the initial column means (A-form sweeps map a constant column to
// itself, so J(X - 1 mu^T) = J(X) - 1 mu^T), and the last sweep accumulates the column sums and
// sums of squares the projection needs, so neither costs an extra pass over the block.
#include "sfg_internal.cuh"
#include "vec.cuh"

namespace {

constexpr int kBlock = 256;
// Tile-shape variants of the sweep, chosen per (K, storage, degree bucket) by sfg_autotune:
// TPI = consecutive row tiles a warp sweeps before its grid-stride jump, MINB = resident CTAs per
// SM requested from the compiler (4 caps registers at 64, 3 at 80).
struct JVariant { int tpi, minb; };
constexpr JVariant kJVariants[] = {{1, 4}, {2, 4}, {4, 4}, {1, 3}, {2, 3}, {4, 3}};
constexpr int kJNumVariants = 6, kJDefault = 1;

// Gaussian entries 2p and 2p+1 of the counter-based generator (see sfg.h): SplitMix64 output
// p + 1 of the stream started in state splitmix64(seed), both Box-Muller branches in FP32 (logf,
// sincospif). The 24-bit angle uniform is exact in FP32.
__device__ __forceinline__ void gaussian_pair(uint64_t s0, uint64_t p, float& x0, float& x1) {
    const uint64_t o = sfg_splitmix64(s0 + p * 0x9E3779B97F4A7C15ull);
    const float u1 = __ull2float_rn((o >> 32) + 1) * 0x1.0p-32f;
    const float u2 = (float)(uint32_t)((o >> 8) & 0xffffffu) * 0x1.0p-24f;
    const float r = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    x0 = r * cs;
    x1 = r * sn;
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

// Seeded block. WEIGHTED = false: partials are the plain column sums and sums of squares (the
// projection statistics when no sweep follows). WEIGHTED = true: partials are sum_i d_i x_ik and
// sum_i d_i, i.e. the D-weighted column means that the first sweep removes. Jacobi sweeps keep
// the D-weighted mean and damp everything else, so removing it (rather than the plain mean) keeps
// the block free of a constant that the final projection would otherwise have to cancel in FP32;
// the two choices differ by a constant vector only, which the projection removes either way.
template <typename T, int LPR, bool WEIGHTED>
__global__ void __launch_bounds__(kBlock) k_init(int32_t n, uint64_t seed, const double* __restrict__ deg,
                                                 T* __restrict__ X, double* __restrict__ part) {
    constexpr int E = Vec<T>::E, K = LPR * E;
    const int lane = threadIdx.x & 31, sub = lane % LPR;
    const int64_t g0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / LPR;
    const int64_t ng = (int64_t)gridDim.x * kBlock / LPR;
    float s1[E], s2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) s1[e] = s2[e] = 0.f;
    const uint64_t s0 = sfg_splitmix64(seed);
    for (int64_t row = g0; row < n; row += ng) {
        float x[E];
#pragma unroll
        for (int e = 0; e < E; e += 2) {
            const uint64_t j = (uint64_t)row * K + sub * E + e;  // even
            gaussian_pair(s0, j >> 1, x[e], x[e + 1]);
        }
        const float d = WEIGHTED ? (float)deg[row] : 1.f;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            x[e] = Vec<T>::round(x[e]);
            if (WEIGHTED) {
                s1[e] = fmaf(d, x[e], s1[e]);
                s2[e] += d;
            } else {
                s1[e] += x[e];
                s2[e] = fmaf(x[e], x[e], s2[e]);
            }
        }
        Vec<T>::store(X + row * K + sub * E, x);
    }
    block_column_partials<LPR, E>(s1, s2, part);
}

template <typename V>
__device__ __forceinline__ V ldmeta(const V* p) {
    return *p;
}

// A chunk of C = max(LPR, 8) consecutive (column, weight) entries of one row, spread over the
// LPR lanes of the row's group (C / LPR per lane). Slots past the row's end hold (row, 0): they
// gather the row itself with weight zero, so the gather loop needs no per-slot predicate.
template <int LPR>
struct Chunk {
    static constexpr int C = LPR >= 8 ? LPR : 8, PER = C / LPR;
    int2 cv[PER];
    __device__ __forceinline__ void load(const int2* __restrict__ colval, int32_t j0, int32_t b,
                                         int32_t self, int sub) {
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int32_t j = j0 + sub + t * LPR;
            cv[t] = j < b ? ldmeta(colval + j) : make_int2(self, 0);
        }
    }
};

// acc += sum over slots [s0, s0 + NS) (slots past the chunk ignored at compile time) of
// w * X[col] for this lane's E columns. All NS gathers are issued before the first is consumed;
// the weights are taken from the chunk at use time, so only the gathered vectors stay live.
template <typename T, int LPR, int NS>
__device__ __forceinline__ void gather_slots(const Chunk<LPR>& ch, int s0, unsigned gm,
                                             const T* __restrict__ Xl, float (&acc)[Vec<T>::E]) {
    constexpr int K = LPR * Vec<T>::E, C = Chunk<LPR>::C;
    uint4 xv[NS];
#pragma unroll
    for (int u = 0; u < NS; ++u) {
        const int slot = s0 + u;
        if (slot < C) {
            const int c = __shfl_sync(gm, ch.cv[slot / LPR].x, slot % LPR, LPR);
            xv[u] = Vec<T>::load_raw(Xl + (int64_t)c * K);
        }
    }
#pragma unroll
    for (int u = 0; u < NS; ++u) {
        const int slot = s0 + u;
        if (slot < C) {
            const float w = __int_as_float(__shfl_sync(gm, ch.cv[slot / LPR].y, slot % LPR, LPR));
            Vec<T>::fma_raw(w, xv[u], acc);
        }
    }
}

// All slots of a chunk that the tile's longest row needs: warp-uniform batches of 2, 4 or 6.
template <typename T, int LPR>
__device__ __forceinline__ void gather_chunk(const Chunk<LPR>& ch, int need, unsigned gm,
                                             const T* __restrict__ Xl, float (&acc)[Vec<T>::E]) {
    constexpr int C = Chunk<LPR>::C;
    if (need <= 2) {
        if (need > 0) gather_slots<T, LPR, 2>(ch, 0, gm, Xl, acc);
    } else if (need <= 4) {
        gather_slots<T, LPR, 4>(ch, 0, gm, Xl, acc);
    } else {
#pragma unroll
        for (int s0 = 0; s0 < C; s0 += 6)
            if (s0 < need) gather_slots<T, LPR, 6>(ch, s0, gm, Xl, acc);
    }
}

// One weighted-Jacobi sweep. A warp owns a tile of GPW = 32 / LPR consecutive rows (one LPR-lane
// group per row) and moves by grid stride over tiles, so all CTAs sweep one moving window of rows
// and the neighbour rows of the window stay in L2. The tile's row_ptr and D^-1 entries come from
// one coalesced load per lane and are handed out by shuffles; each group holds its row's first
// chunk of (column, weight) entries. The next tile's metadata is loaded before this tile's
// gathers are issued and its chunks right after, so one gather round is the only exposed latency
// per tile. Gathers go in warp-uniform batches sized by the tile's longest row. Rows with more
// than hmax entries are left to the heavy-row kernels below (their group idles through the tile
// and stores nothing), so one hub row cannot serialise a warp for the whole sweep.
template <typename T, int LPR, bool SUB_MU, bool STATS, int TPI, int MINB>
__global__ void __launch_bounds__(kBlock, MINB)
    k_jacobi(int32_t n, int32_t hmax, const int32_t* __restrict__ row_ptr, const int2* __restrict__ colval,
             const float* __restrict__ coef, float a_self, const T* __restrict__ X,
             T* __restrict__ Y, const float* __restrict__ mu, double* __restrict__ part) {
    constexpr int E = Vec<T>::E, K = LPR * E, GPW = 32 / LPR, C = Chunk<LPR>::C;
    const int lane = threadIdx.x & 31, grp = lane / LPR, sub = lane % LPR;
    const unsigned gm = group_mask<LPR>(lane);
    const int32_t wid = (int32_t)((blockIdx.x * kBlock + threadIdx.x) >> 5);
    const int32_t nw = (int32_t)(gridDim.x * (kBlock / 32));
    const int32_t ntiles = (n + GPW - 1) / GPW;
    const T* __restrict__ Xl = X + sub * E;
    // tile order of this warp: TPI consecutive tiles, then a jump over the other warps' tiles
    auto next_tile = [&](int32_t t) {
        return (t + 1) % TPI != 0 ? t + 1 : t + 1 + (nw - 1) * TPI;
    };

    float m[E], s1[E], s2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        m[e] = SUB_MU ? mu[sub * E + e] : 0.f;
        s1[e] = s2[e] = 0.f;
    }
    // Metadata of tile t, one value per lane: lo = row_ptr[r0 + lane], hi = row_ptr[r0 + lane + 1]
    // (both clamped at n; hi only when GPW = 32), cf = D^-1 of row r0 + lane.
    struct Meta { int32_t lo, hi; float cf; };
    // this group's row bounds in tile metadata mt; a heavy row gets b = a - 1 (no entries, and
    // deg < 0 marks it as not stored here)
    auto bounds = [&](const Meta& mt, int32_t& a, int32_t& b) {
        a = __shfl_sync(0xffffffffu, mt.lo, grp);
        b = GPW == 32 ? mt.hi : __shfl_sync(0xffffffffu, mt.lo, grp + 1);
        if (b - a > hmax) b = a - 1;
    };
    auto load_meta = [&](int32_t t) {
        Meta mt{0, 0, 0.f};
        const int32_t r = t * GPW + lane;
        if (t < ntiles && lane <= GPW) mt.lo = ldmeta(row_ptr + min(r, n));
        if (GPW == 32 && t < ntiles) mt.hi = ldmeta(row_ptr + min(r + 1, n));
        if (t < ntiles && lane < GPW && r < n) mt.cf = ldmeta(coef + r);
        return mt;
    };
    // The rows of tile t: gathers, then mid() (work to overlap with the update), the update, the
    // store and the projection statistics.
    auto row_tile = [&](int32_t t, const Chunk<LPR>& ch, int32_t a, int32_t b, float cp, auto&& mid) {
        const int32_t r = t * GPW + grp;
        const int32_t self = r < n ? r : 0;
        const int32_t deg = b - a;
        const bool live = r < n && deg >= 0;
        const int32_t maxdeg = __reduce_max_sync(0xffffffffu, deg);
        float acc[E];
        const uint4 xr = Vec<T>::load_raw(Xl + (int64_t)self * K);  // widened at use
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;
        gather_chunk<T, LPR>(ch, min(maxdeg, C), gm, Xl, acc);
        for (int32_t j0 = C; j0 < maxdeg; j0 += C) {  // rows longer than one chunk
            Chunk<LPR> cx;
            cx.load(colval, a + j0, b, self, sub);
            gather_chunk<T, LPR>(cx, min(maxdeg - j0, C), gm, Xl, acc);
        }
        mid();
        if (live) {
            float xs[E], y[E];
            Vec<T>::unpack(xr, xs);
            if (deg > 0) {
#pragma unroll
                for (int e = 0; e < E; ++e) y[e] = fmaf(cp, acc[e], a_self * xs[e]) - m[e];
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) y[e] = xs[e] - m[e];
            }
            Vec<T>::store(Y + (int64_t)r * K + sub * E, y);
            if (STATS)
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const float q = Vec<T>::round(y[e]);
                    s1[e] += q;
                    s2[e] = fmaf(q, q, s2[e]);
                }
        }
    };

    if constexpr (LPR <= 8) {
        // Three tiles are in flight: t is gathered, the next tile's chunk is loaded, and the metadata
        // of the one after it is loaded. The next tile's bounds come from metadata issued one gather
        // round earlier and its chunk is issued before this tile's gathers, so each tile exposes one
        // gather round and nothing else.
        int32_t t = wid * TPI;
        const Meta mt0 = load_meta(t);
        Meta mt1 = load_meta(next_tile(t));
        int32_t a, b;
        bounds(mt0, a, b);
        float cp = __shfl_sync(0xffffffffu, mt0.cf, grp);
        Chunk<LPR> ch;
        ch.load(colval, a, b, min(t * GPW + grp, n - 1), sub);
        while (t < ntiles) {
            const int32_t t1 = next_tile(t);
            int32_t a1, b1;
            bounds(mt1, a1, b1);
            Chunk<LPR> ch1;
            ch1.load(colval, a1, b1, min(t1 * GPW + grp, n - 1), sub);
            const Meta mt2 = load_meta(next_tile(t1));
            row_tile(t, ch, a, b, cp, [] {});
            t = t1;
            ch = ch1;
            a = a1;
            b = b1;
            cp = __shfl_sync(0xffffffffu, mt1.cf, grp);
            mt1 = mt2;
        }
    } else {
        // LPR = 16 (two rows per tile): two tiles in flight, t is gathered while the next tile's
        // metadata is loaded and its chunk follows the gather round (measured faster at this shape).
        int32_t t = wid * TPI;
        Meta mt = load_meta(t);
        int32_t a, b;
        bounds(mt, a, b);
        Chunk<LPR> ch;
        ch.load(colval, a, b, min(t * GPW + grp, n - 1), sub);
        for (; t < ntiles;) {
            const int32_t t1 = next_tile(t);
            const Meta mt1 = load_meta(t1);
            const int32_t a0 = a, b0 = b;
            const Chunk<LPR> ch0 = ch;
            row_tile(t, ch0, a0, b0, __shfl_sync(0xffffffffu, mt.cf, grp), [&] {
                bounds(mt1, a, b);
                ch.load(colval, a, b, min(t1 * GPW + grp, n - 1), sub);
            });
            mt = mt1;
            t = t1;
        }
    }
    if (STATS) block_column_partials<LPR, E>(s1, s2, part);
}

// Rows longer than kHeavy entries (the hubs of power-law graphs) are swept apart from the tiles:
// each is cut into segments of kSeg consecutive entries, one lane group per segment forms the
// partial sum of w * X[col] over its segment (k_heavy_part), and one group per row adds the row's
// partials in segment order and applies the update (k_heavy_final). The segmentation is fixed per
// graph, so the result does not depend on the schedule. The lists are built once per graph.
constexpr int32_t kHeavy = SFG_HEAVY_ROW, kSeg = SFG_HEAVY_SEG;
constexpr int kHeavyGrid = 64;  // CTAs of k_heavy_final: its statistics take as many part slots

template <typename T, int LPR>
__global__ void __launch_bounds__(kBlock) k_heavy_part(int64_t nseg, const int4* __restrict__ seg,
                                                       const int2* __restrict__ colval,
                                                       const T* __restrict__ X,
                                                       float* __restrict__ partial) {
    constexpr int E = Vec<T>::E, K = LPR * E, GPW = 32 / LPR, C = Chunk<LPR>::C;
    const int lane = threadIdx.x & 31, grp = lane / LPR, sub = lane % LPR;
    const unsigned gm = group_mask<LPR>(lane);
    const int64_t w0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int64_t nw = (int64_t)gridDim.x * (kBlock / 32);
    const T* __restrict__ Xl = X + sub * E;
    for (int64_t s0 = w0 * GPW; s0 < nseg; s0 += nw * GPW) {
        const int64_t sid = s0 + grp;
        const bool live = sid < nseg;
        const int4 sg = live ? seg[sid] : make_int4(0, 0, 0, 0);  // (row, begin, end, -)
        float acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;
        // the same trip count for every group: slots past a segment's end gather the row itself
        // with weight zero
#pragma unroll 1
        for (int32_t j0 = 0; j0 < kSeg; j0 += C) {
            Chunk<LPR> ch;
            ch.load(colval, sg.y + j0, sg.z, sg.x, sub);
#pragma unroll
            for (int q = 0; q < C; q += 8) gather_slots<T, LPR, 8>(ch, q, gm, Xl, acc);
        }
        if (live) {
            float* pr = partial + sid * K + sub * E;
#pragma unroll
            for (int e = 0; e < E; e += 4)
                *reinterpret_cast<float4*>(pr + e) = make_float4(acc[e], acc[e + 1], acc[e + 2], acc[e + 3]);
        }
    }
}

template <typename T, int LPR, bool SUB_MU, bool STATS>
__global__ void __launch_bounds__(kBlock) k_heavy_final(int32_t nh, const int32_t* __restrict__ hrow,
                                                        const int32_t* __restrict__ hsoff,
                                                        const float* __restrict__ partial,
                                                        const float* __restrict__ coef, float a_self,
                                                        const T* __restrict__ X, T* __restrict__ Y,
                                                        const float* __restrict__ mu,
                                                        double* __restrict__ part) {
    constexpr int E = Vec<T>::E, K = LPR * E;
    const int sub = (threadIdx.x & 31) % LPR;
    const int64_t g0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / LPR;
    const int64_t ng = (int64_t)gridDim.x * kBlock / LPR;
    float m[E], s1[E], s2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        m[e] = SUB_MU ? mu[sub * E + e] : 0.f;
        s1[e] = s2[e] = 0.f;
    }
    for (int64_t h = g0; h < nh; h += ng) {
        const int32_t r = hrow[h];
        float acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;
        for (int32_t sid = hsoff[h]; sid < hsoff[h + 1]; ++sid) {
            const float* pr = partial + (int64_t)sid * K + sub * E;
#pragma unroll
            for (int e = 0; e < E; e += 4) {
                const float4 q = *reinterpret_cast<const float4*>(pr + e);
                acc[e] += q.x;
                acc[e + 1] += q.y;
                acc[e + 2] += q.z;
                acc[e + 3] += q.w;
            }
        }
        float xs[E], y[E];
        Vec<T>::unpack(Vec<T>::load_raw(X + (int64_t)r * K + sub * E), xs);
        const float cp = coef[r];
#pragma unroll
        for (int e = 0; e < E; ++e) y[e] = fmaf(cp, acc[e], a_self * xs[e]) - m[e];
        Vec<T>::store(Y + (int64_t)r * K + sub * E, y);
        if (STATS)
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const float q = Vec<T>::round(y[e]);
                s1[e] += q;
                s2[e] = fmaf(q, q, s2[e]);
            }
    }
    if (STATS) block_column_partials<LPR, E>(s1, s2, part);
}

__global__ void k_heavy_mark(int32_t n, const int32_t* __restrict__ row_ptr, int32_t* __restrict__ heavy,
                             int32_t* __restrict__ nseg, int* __restrict__ count) {
    int c = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = row_ptr[r + 1] - row_ptr[r];
        heavy[r] = d > kHeavy;
        nseg[r] = d > kHeavy ? (d + kSeg - 1) / kSeg : 0;
        c += d > kHeavy;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

__global__ void k_heavy_fill(int32_t n, const int32_t* __restrict__ row_ptr, const int64_t* __restrict__ hoff,
                             const int64_t* __restrict__ soff, int32_t* __restrict__ hrow,
                             int32_t* __restrict__ hsoff, int4* __restrict__ seg) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        if (r == 0) hsoff[hoff[n]] = (int32_t)soff[n];
        if (hoff[r + 1] == hoff[r]) continue;
        const int64_t h = hoff[r];
        hrow[h] = (int32_t)r;
        hsoff[h] = (int32_t)soff[r];
        const int32_t a = row_ptr[r], b = row_ptr[r + 1];
        int64_t o = soff[r];
        for (int32_t j = a; j < b; j += kSeg) seg[o++] = make_int4((int32_t)r, j, min(j + kSeg, b), 0);
    }
}

// For each heavy row h: (row, colour, first entry, end entry).
__global__ void k_heavy_gather(int32_t nh, const int32_t* __restrict__ hrow, const int32_t* __restrict__ color,
                               const int32_t* __restrict__ row_ptr, int32_t* __restrict__ out) {
    const int32_t h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= nh) return;
    const int32_t r = hrow[h];
    out[4 * h] = r;
    out[4 * h + 1] = color[r];
    out[4 * h + 2] = row_ptr[r];
    out[4 * h + 3] = row_ptr[r + 1];
}

// Heavy-row lists of L (a cache of the graph, built with it).
sfg_status heavy_prepare(sfg_ctx* ctx, const sfg_graph* Lc) {
    sfg_graph* L = const_cast<sfg_graph*>(Lc);
    if (L->hv_n >= 0) return SFG_OK;
    const int32_t n = L->n;
    if (n == 0) {
        L->hv_n = 0;
        return SFG_OK;
    }
    Scratch s(ctx);
    int32_t *heavy, *nseg;
    int64_t *hoff, *soff;
    int* count;
    SFG_TRY(s.get(&heavy, (size_t)n));
    SFG_TRY(s.get(&nseg, (size_t)n));
    SFG_TRY(s.get(&count, 1));
    SFG_CUDA(ctx, cudaMemsetAsync(count, 0, sizeof(int), ctx->stream));
    const int g = sfg_grid(ctx, (const void*)k_heavy_mark, kBlock, 0, n);
    k_heavy_mark<<<g, kBlock, 0, ctx->stream>>>(n, L->row_ptr, heavy, nseg, count);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_heavy_mark");
    int hcount = 0;
    SFG_CUDA(ctx, cudaMemcpyAsync(&hcount, count, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (hcount == 0) {  // the common case on meshes: one pass over row_ptr, one readback
        L->hv_nseg = 0;
        L->hv_n = 0;
        return SFG_OK;
    }
    SFG_TRY(s.get(&hoff, (size_t)n + 1));
    SFG_TRY(s.get(&soff, (size_t)n + 1));
    SFG_TRY(sfg_scan_i32(ctx, heavy, hoff, n));
    SFG_TRY(sfg_scan_i32(ctx, nseg, soff, n));
    int64_t nh = 0, ns = 0;
    SFG_TRY(sfg_read_i64(ctx, hoff + n, &nh));
    SFG_TRY(sfg_read_i64(ctx, soff + n, &ns));
    if (nh > 0) {
        int32_t *hrow = nullptr, *hsoff = nullptr;
        int4* seg = nullptr;
        sfg_status st = sfg_alloc(ctx, (void**)&hrow, sizeof(int32_t) * nh);
        if (st == SFG_OK) st = sfg_alloc(ctx, (void**)&hsoff, sizeof(int32_t) * (nh + 1));
        if (st == SFG_OK) st = sfg_alloc(ctx, (void**)&seg, sizeof(int4) * ns);
        if (st != SFG_OK) {
            for (void* q : {(void*)hrow, (void*)hsoff, (void*)seg})
                if (q) sfg_free(ctx, q);
            return st;
        }
        L->hv_rows = hrow;  // owned by the graph from here on
        L->hv_soff = hsoff;
        L->hv_seg = seg;
        k_heavy_fill<<<g, kBlock, 0, ctx->stream>>>(n, L->row_ptr, hoff, soff, hrow, hsoff, seg);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_heavy_fill");
    }
    L->hv_nseg = ns;
    L->hv_n = (int32_t)nh;
    return SFG_OK;
}

// One colour class of a multicolour Gauss-Seidel sweep (Sec. 3.2 relaxes L x = 0 with
// Gauss-Seidel): rows[0, cnt) are pairwise non-adjacent, so each is updated in place from the
// current values of its neighbours, x_p <- (1 - omega) x_p + (omega / D(p,p)) (A x)_p, which is the
// sequential sweep restricted to this class. Same group layout and gathers as the Jacobi sweep;
// the tile's rows come from the class list, one tile at a time. X is read and written through
// plain pointers (rows of this class are written, only rows of other classes are gathered).
template <typename T, int LPR>
__global__ void __launch_bounds__(kBlock, 4)
    k_gs(int32_t cnt, const int32_t* __restrict__ rows, const int32_t* __restrict__ row_ptr,
         const int2* __restrict__ colval, const float* __restrict__ coef, float a_self, T* X,
         int32_t hmax) {
    constexpr int E = Vec<T>::E, K = LPR * E, GPW = 32 / LPR, C = Chunk<LPR>::C;
    const int lane = threadIdx.x & 31, grp = lane / LPR, sub = lane % LPR;
    const unsigned gm = group_mask<LPR>(lane);
    const int32_t wid = (int32_t)((blockIdx.x * kBlock + threadIdx.x) >> 5);
    const int32_t nw = (int32_t)(gridDim.x * (kBlock / 32));
    const int32_t ntiles = (cnt + GPW - 1) / GPW;
    const T* Xl = X + sub * E;
    for (int32_t t = wid; t < ntiles; t += nw) {
        const int32_t i = t * GPW + lane;
        int32_t r = -1, lo = 0, hi = 0;
        float cf = 0.f;
        if (lane < GPW && i < cnt) {
            r = rows[i];
            lo = row_ptr[r];
            hi = row_ptr[r + 1];
            cf = coef[r];
            if (hi - lo > hmax) hi = lo - 1;  // updated by the heavy-row kernels of this class
        }
        const int32_t row = __shfl_sync(0xffffffffu, r, grp);
        const int32_t a = __shfl_sync(0xffffffffu, lo, grp);
        const int32_t b = __shfl_sync(0xffffffffu, hi, grp);
        const float cp = __shfl_sync(0xffffffffu, cf, grp);
        const bool live = row >= 0;
        const int32_t first = __shfl_sync(0xffffffffu, r, 0);  // all lanes: the tile's first row
        const int32_t self = live ? row : first;
        const int32_t deg = b - a;
        const int32_t maxdeg = __reduce_max_sync(0xffffffffu, deg);
        Chunk<LPR> ch;
        ch.load(colval, a, b, self, sub);
        float acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;
        gather_chunk<T, LPR>(ch, min(maxdeg, C), gm, Xl, acc);
        for (int32_t j0 = C; j0 < maxdeg; j0 += C) {
            Chunk<LPR> cx;
            cx.load(colval, a + j0, b, self, sub);
            gather_chunk<T, LPR>(cx, min(maxdeg - j0, C), gm, Xl, acc);
        }
        if (live && deg > 0) {
            T* xp = X + (int64_t)self * K + sub * E;
            float xs[E], y[E];
            Vec<T>::load(xp, xs);
#pragma unroll
            for (int e = 0; e < E; ++e) y[e] = fmaf(cp, acc[e], a_self * xs[e]);
            Vec<T>::store(xp, y);
        }
    }
}

// The heavy rows of one colour class, in place: row h adds its segments' partials (segment ids
// soff[h] - base ... soff[h + 1] - base of this class's partial array) and applies the update of
// k_gs. Rows of one class are not adjacent, so the partials read only rows of other classes.
template <typename T, int LPR>
__global__ void __launch_bounds__(kBlock) k_heavy_final_gs(int32_t nh, const int32_t* __restrict__ hrow,
                                                           const int32_t* __restrict__ hsoff, int64_t base,
                                                           const float* __restrict__ partial,
                                                           const float* __restrict__ coef, float a_self,
                                                           T* X) {
    constexpr int E = Vec<T>::E, K = LPR * E;
    const int sub = (threadIdx.x & 31) % LPR;
    const int64_t g0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / LPR;
    const int64_t ng = (int64_t)gridDim.x * kBlock / LPR;
    for (int64_t h = g0; h < nh; h += ng) {
        const int32_t r = hrow[h];
        float acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;
        for (int64_t sid = hsoff[h] - base; sid < hsoff[h + 1] - base; ++sid) {
            const float* pr = partial + sid * K + sub * E;
#pragma unroll
            for (int e = 0; e < E; e += 4) {
                const float4 q = *reinterpret_cast<const float4*>(pr + e);
                acc[e] += q.x;
                acc[e + 1] += q.y;
                acc[e + 2] += q.z;
                acc[e + 3] += q.w;
            }
        }
        T* xp = X + (int64_t)r * K + sub * E;
        float xs[E], y[E];
        Vec<T>::load(xp, xs);
        const float cp = coef[r];
#pragma unroll
        for (int e = 0; e < E; ++e) y[e] = fmaf(cp, acc[e], a_self * xs[e]);
        Vec<T>::store(xp, y);
    }
}

// Heavy rows of L grouped by colour class (a cache of the graph, built on the first
// Gauss-Seidel smoothing): rows sorted by (colour, id), their segments in that order, and the
// per-colour offsets of both on the host.
sfg_status gs_heavy_prepare(sfg_ctx* ctx, const sfg_graph* Lc) {
    sfg_graph* L = const_cast<sfg_graph*>(Lc);
    if (L->gh_ready) return SFG_OK;
    const int ncol = (int)L->gs_off.size() - 1;
    L->gh_coff.assign((size_t)std::max(ncol, 0) + 1, 0);
    L->gh_scoff.assign((size_t)std::max(ncol, 0) + 1, 0);
    const int32_t nh = std::max(L->hv_n, 0);
    if (nh == 0 || ncol <= 0) {
        L->gh_ready = true;
        return SFG_OK;
    }
    std::vector<int32_t> h4((size_t)4 * nh);
    {
        Scratch s(ctx);
        int32_t* dev4;
        SFG_TRY(s.get(&dev4, (size_t)4 * nh));
        k_heavy_gather<<<ceil_div_u(nh, kBlock), kBlock, 0, ctx->stream>>>(nh, L->hv_rows, L->gs_color,
                                                                            L->row_ptr, dev4);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_heavy_gather");
        SFG_CUDA(ctx, cudaMemcpyAsync(h4.data(), dev4, sizeof(int32_t) * 4 * nh, cudaMemcpyDeviceToHost,
                                      ctx->stream));
        SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    // stable by colour: hv_rows are in id order, so each class keeps increasing ids
    std::vector<int32_t> ord(nh);
    for (int32_t h = 0; h < nh; ++h) ord[h] = h;
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int32_t a, int32_t b) { return h4[4 * a + 1] < h4[4 * b + 1]; });
    std::vector<int32_t> grows(nh), gsoff((size_t)nh + 1);
    std::vector<int64_t> ccount((size_t)ncol, 0), scount((size_t)ncol, 0);
    std::vector<int4> gseg;
    for (int32_t k = 0; k < nh; ++k) {
        const int32_t h = ord[k], r = h4[4 * h], c = h4[4 * h + 1], lo = h4[4 * h + 2], hi = h4[4 * h + 3];
        grows[k] = r;
        gsoff[k] = (int32_t)gseg.size();
        for (int32_t j = lo; j < hi; j += kSeg) gseg.push_back(make_int4(r, j, std::min(j + kSeg, hi), 0));
        ccount[c] += 1;
        scount[c] += (hi - lo + kSeg - 1) / kSeg;
    }
    gsoff[nh] = (int32_t)gseg.size();
    for (int c = 0; c < ncol; ++c) {
        L->gh_coff[c + 1] = L->gh_coff[c] + ccount[c];
        L->gh_scoff[c + 1] = L->gh_scoff[c] + scount[c];
    }
    int32_t *drows = nullptr, *dsoff = nullptr;
    int4* dseg = nullptr;
    sfg_status st = sfg_alloc(ctx, (void**)&drows, sizeof(int32_t) * nh);
    if (st == SFG_OK) st = sfg_alloc(ctx, (void**)&dsoff, sizeof(int32_t) * (nh + 1));
    if (st == SFG_OK) st = sfg_alloc(ctx, (void**)&dseg, sizeof(int4) * gseg.size());
    if (st != SFG_OK) {
        for (void* q : {(void*)drows, (void*)dsoff, (void*)dseg})
            if (q) sfg_free(ctx, q);
        return st;
    }
    L->gh_rows = drows;
    L->gh_soff = dsoff;
    L->gh_seg = dseg;
    SFG_CUDA(ctx, cudaMemcpyAsync(drows, grows.data(), sizeof(int32_t) * nh, cudaMemcpyHostToDevice,
                                  ctx->stream));
    SFG_CUDA(ctx, cudaMemcpyAsync(dsoff, gsoff.data(), sizeof(int32_t) * (nh + 1), cudaMemcpyHostToDevice,
                                  ctx->stream));
    SFG_CUDA(ctx, cudaMemcpyAsync(dseg, gseg.data(), sizeof(int4) * gseg.size(), cudaMemcpyHostToDevice,
                                  ctx->stream));
    SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // the host arrays go out of scope
    L->gh_ready = true;
    return SFG_OK;
}

__global__ void k_fill(int k, float v, float* __restrict__ p) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) p[i] = v;
}

// Per-block column sums and sums of squares of a stored block (values as stored).
template <typename T, int LPR>
__global__ void __launch_bounds__(kBlock) k_col_stats(int32_t n, const T* __restrict__ X,
                                                      double* __restrict__ part) {
    constexpr int E = Vec<T>::E, K = LPR * E;
    const int sub = (threadIdx.x & 31) % LPR;
    float s1[E], s2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) s1[e] = s2[e] = 0.f;
    const int64_t g0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / LPR;
    const int64_t gs = (int64_t)gridDim.x * kBlock / LPR;
    for (int64_t r = g0; r < n; r += gs) {
        float x[E];
        Vec<T>::load(X + r * K + sub * E, x);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            s1[e] += x[e];
            s2[e] = fmaf(x[e], x[e], s2[e]);
        }
    }
    block_column_partials<LPR, E>(s1, s2, part);
}

// Fold the per-block partials (FP64): one CTA per column, each thread sums a fixed stride of
// blocks, then a fixed-shape tree, so the result does not depend on scheduling.
// proj = 0: mean only (mu = S1 / n). proj = 1: mean and scale = 1 / RMS of the centred column
// (1 if the column is zero). proj = 2: D-weighted mean S1 / S2 of k_init<WEIGHTED>.
__global__ void __launch_bounds__(kBlock) k_finalize(const double* __restrict__ part, int nblocks,
                                                     int K, int32_t n, int proj,
                                                     float* __restrict__ mean,
                                                     float* __restrict__ scale) {
    __shared__ double r1[kBlock], r2[kBlock];
    const int k = blockIdx.x;
    double s1 = 0.0, s2 = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kBlock) {
        s1 += part[(size_t)b * 2 * K + k];
        s2 += part[(size_t)b * 2 * K + K + k];
    }
    r1[threadIdx.x] = s1;
    r2[threadIdx.x] = s2;
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            r1[threadIdx.x] += r1[threadIdx.x + w];
            r2[threadIdx.x] += r2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (proj == 2) {  // D-weighted mean: sum d x / sum d
            mean[k] = r2[0] > 0.0 ? (float)(r1[0] / r2[0]) : 0.f;
            return;
        }
        const double mu = r1[0] / (double)n;
        mean[k] = (float)mu;
        if (proj) {
            const double var = r2[0] / (double)n - mu * mu;
            const double rms = var > 0.0 ? sqrt(var) : 0.0;
            scale[k] = rms > 0.0 ? (float)(1.0 / rms) : 1.0f;
        }
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

// c_p = omega * (1 / D(p,p)) with the reciprocal formed once per graph in FP64; 0 if D(p,p) = 0.
__global__ void k_coef(int32_t n, const double* __restrict__ invdeg, double omega,
                       float* __restrict__ coef) {
    for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kBlock)
        coef[p] = (float)(omega * invdeg[p]);
}

// ------------------------------------------------------------------------------------------------
// Batched embedding of a disjoint union of graphs (rows of graph g are [node_off[g],
// node_off[g+1]) ). Sweeps need nothing per graph; the seeded block, its mean removal and the
// projection statistics are per graph, so every graph gets exactly the block and statistics it
// would get alone (up to FP32 summation order).
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ int32_t graph_of(const int32_t* __restrict__ off, int ng, int64_t r) {
    int lo = 0, hi = ng;  // last g with off[g] <= r
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= r) lo = mid; else hi = mid;
    }
    return lo;
}

template <typename T, int LPR>
__global__ void __launch_bounds__(kBlock) k_init_batched(int32_t n, uint64_t seed,
                                                         const int32_t* __restrict__ node_off,
                                                         int ng, const int32_t* __restrict__ orig_local,
                                                         T* __restrict__ X) {
    constexpr int E = Vec<T>::E, K = LPR * E;
    const int lane = threadIdx.x & 31, sub = lane % LPR;
    const int64_t g0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / LPR;
    const int64_t ng_ = (int64_t)gridDim.x * kBlock / LPR;
    const uint64_t s0 = sfg_splitmix64(seed);
    for (int64_t row = g0; row < n; row += ng_) {
        const int64_t local = orig_local ? (int64_t)orig_local[row]
                                         : row - node_off[graph_of(node_off, ng, row)];
        float x[E];
#pragma unroll
        for (int e = 0; e < E; e += 2) {
            const uint64_t j = (uint64_t)local * K + sub * E + e;
            gaussian_pair(s0, j >> 1, x[e], x[e + 1]);
        }
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = Vec<T>::round(x[e]);
        Vec<T>::store(X + row * K + sub * E, x);
    }
}

// Per-graph column sums and sums of squares (FP64) of X. Every graph's rows are cut into
// kSegSlices equal contiguous slices, one CTA per (graph, slice): each LPR-lane group folds 64-row
// chunks in FP32 (the chunk's rows loaded 8 at a time, accumulated in row order) into FP64, then a
// fixed-shape tree across the CTA gives the slice's partials; k_seg_reduce adds a graph's slices in
// slice order. The partition does not depend on the launch, so the sums are deterministic.
// deg != NULL: sums of d_i x_ik and of d_i instead (the D-weighted means, see k_init).
constexpr int kSegSlices = 32;

template <typename T, int LPR>
__global__ void __launch_bounds__(kBlock) k_seg_stats(const T* __restrict__ X,
                                                      const int32_t* __restrict__ node_off,
                                                      const double* __restrict__ deg,
                                                      double* __restrict__ part) {
    constexpr int E = Vec<T>::E, K = LPR * E, GPB = kBlock / LPR, NB = 8;
    __shared__ double red[kBlock / 32][2 * K];
    const int g = blockIdx.x / kSegSlices, q = blockIdx.x % kSegSlices;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, sub = lane % LPR;
    const int64_t g0 = node_off[g], rows = node_off[g + 1] - g0;
    const int64_t r0 = g0 + rows * q / kSegSlices, r1 = g0 + rows * (q + 1) / kSegSlices;
    double d1[E], d2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) d1[e] = d2[e] = 0.0;
    for (int64_t base = r0 + threadIdx.x / LPR; base < r1; base += (int64_t)GPB * 64) {
        float f1[E], f2[E];
#pragma unroll
        for (int e = 0; e < E; ++e) f1[e] = f2[e] = 0.f;
        for (int i0 = 0; i0 < 64; i0 += NB) {
            if (base + (int64_t)i0 * GPB >= r1) break;
            float x[NB][E], d[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) {  // all loads of the batch before any use
                const int64_t r = base + (int64_t)(i0 + b) * GPB;
                const bool ok = r < r1;
                if (ok) Vec<T>::load(X + r * K + sub * E, x[b]);
                d[b] = ok && deg ? (float)deg[r] : 0.f;
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (base + (int64_t)(i0 + b) * GPB >= r1) break;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (deg) {
                        f1[e] = fmaf(d[b], x[b][e], f1[e]);
                        f2[e] += d[b];
                    } else {
                        f1[e] += x[b][e];
                        f2[e] = fmaf(x[b][e], x[b][e], f2[e]);
                    }
                }
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            d1[e] += f1[e];
            d2[e] += f2[e];
        }
    }
#pragma unroll
    for (int o = LPR; o < 32; o <<= 1)
#pragma unroll
        for (int e = 0; e < E; ++e) {
            d1[e] += __shfl_xor_sync(0xffffffffu, d1[e], o);
            d2[e] += __shfl_xor_sync(0xffffffffu, d2[e], o);
        }
    if (lane < LPR)
#pragma unroll
        for (int e = 0; e < E; ++e) {
            red[warp][sub * E + e] = d1[e];
            red[warp][K + sub * E + e] = d2[e];
        }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * K; t += kBlock) {
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) acc += red[w][t];
        part[(size_t)blockIdx.x * 2 * K + t] = acc;
    }
}

// stats[g][t] = sum over the slices of graph g, in slice order, of their partials
__global__ void k_seg_reduce(int ng, int K2, const double* __restrict__ part,
                             double* __restrict__ stats) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)ng * K2) return;
    const int64_t g = i / K2, t = i % K2;
    double acc = 0.0;
    for (int q = 0; q < kSegSlices; ++q) acc += part[((size_t)g * kSegSlices + q) * K2 + t];
    stats[i] = acc;
}

// mean[g][k], scale[g][k] (scale = 1 / RMS of the centred column, 1 if zero) from the stats.
// weighted: mean = s1 / s2 of k_seg_stats with degrees (no scale).
__global__ void k_seg_finalize(const double* __restrict__ stats, const int32_t* __restrict__ node_off,
                               int ng, int K, int weighted, float* __restrict__ mean,
                               float* __restrict__ scale) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)ng * K) return;
    const int g = (int)(i / K), k = (int)(i % K);
    const double n = (double)(node_off[g + 1] - node_off[g]);
    const double s1 = stats[(size_t)g * 2 * K + k], s2 = stats[(size_t)g * 2 * K + K + k];
    if (weighted) {
        mean[i] = s2 > 0.0 ? (float)(s1 / s2) : 0.f;
        return;
    }
    const double mu = n > 0 ? s1 / n : 0.0;
    mean[i] = (float)mu;
    if (scale) {
        const double var = n > 0 ? s2 / n - mu * mu : 0.0;
        const double rms = var > 0.0 ? sqrt(var) : 0.0;
        scale[i] = rms > 0.0 ? (float)(1.0 / rms) : 1.0f;
    }
}

template <typename T, int LPR>
__global__ void __launch_bounds__(kBlock) k_center_batched(int32_t n, const int32_t* __restrict__ node_off,
                                                           int ng, const float* __restrict__ mean,
                                                           T* __restrict__ X) {
    constexpr int E = Vec<T>::E, K = LPR * E;
    const int lane = threadIdx.x & 31, sub = lane % LPR;
    const int64_t g0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / LPR;
    const int64_t ng_ = (int64_t)gridDim.x * kBlock / LPR;
    for (int64_t row = g0; row < n; row += ng_) {
        const int g = graph_of(node_off, ng, row);
        float x[E];
        Vec<T>::load(X + row * K + sub * E, x);
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] -= mean[(size_t)g * K + sub * E + e];
        Vec<T>::store(X + row * K + sub * E, x);
    }
}

template <typename T, int LPR>
struct Smoother {
    using Elem = T;
    static constexpr int E = Vec<T>::E, K = LPR * E;

    template <bool A, bool B>
    static void* kern() {
        return (void*)k_jacobi<T, LPR, A, B, kJVariants[kJDefault].tpi, kJVariants[kJDefault].minb>;
    }
    static void* plain_kern(int v) {  // the tuned variants of the plain sweep
        switch (v) {
            case 0: return (void*)k_jacobi<T, LPR, false, false, 1, 4>;
            case 2: return (void*)k_jacobi<T, LPR, false, false, 4, 4>;
            case 3: return (void*)k_jacobi<T, LPR, false, false, 1, 3>;
            case 4: return (void*)k_jacobi<T, LPR, false, false, 2, 3>;
            case 5: return (void*)k_jacobi<T, LPR, false, false, 4, 3>;
            default: return (void*)k_jacobi<T, LPR, false, false, 2, 4>;
        }
    }

    static int grid_jacobi(sfg_ctx* ctx, int32_t n) {
        return sfg_grid(ctx, kern<false, false>(), kBlock, 0, (int64_t)n * LPR);
    }

    // Statistics slots a sweep of L with `grid` tile CTAs writes (the heavy rows add theirs).
    static int part_slots(const sfg_graph* L, int grid) {
        return grid + (L->hv_n > 0 ? kHeavyGrid : 0);
    }

    static sfg_status sweep(sfg_ctx* ctx, const sfg_graph* L, const float* coef, float a_self,
                            const T* X, T* Y, const float* mu, double* part, bool sub_mu,
                            bool stats, int grid) {
        const int32_t n = L->n;
        SFG_TRY(heavy_prepare(ctx, L));
        const int32_t hmax = L->hv_n > 0 ? kHeavy : INT32_MAX;
        void* k = sub_mu ? (stats ? kern<true, true>() : kern<true, false>())
                         : (stats ? kern<false, true>() : kern<false, false>());
        int g = grid;
        if (!sub_mu && !stats) {  // the plain sweep takes the tuned tile shape, if any
            const int v = sfg_tuned_variant(ctx, K, Vec<T>::E == 4 ? SFG_F32 : SFG_BF16, L);
            if (v >= 0 && v != kJDefault) {
                k = plain_kern(v);
                g = sfg_grid(ctx, k, kBlock, 0, (int64_t)n * LPR);
            }
        }
        void* args[] = {(void*)&n, (void*)&hmax, (void*)&L->row_ptr, (void*)&L->colval, (void*)&coef,
                        (void*)&a_self, (void*)&X, (void*)&Y, (void*)&mu, (void*)&part};
        sfg_tic(ctx, "jacobi");
        ++ctx->launches;
        const cudaError_t e = cudaLaunchKernel(k, dim3(g), dim3(kBlock), args, 0, ctx->stream);
        sfg_toc(ctx);
        if (e != cudaSuccess) return sfg_cuda_fail(ctx, e, "k_jacobi");
        if (L->hv_n > 0) {
            Scratch sc(ctx);
            float* partial;
            SFG_TRY(sc.get(&partial, (size_t)L->hv_nseg * K));
            const int gp = sfg_grid(ctx, (const void*)k_heavy_part<T, LPR>, kBlock, 0,
                                    L->hv_nseg * LPR);
            sfg_tic(ctx, "jacobi_heavy");
            k_heavy_part<T, LPR><<<gp, kBlock, 0, ctx->stream>>>(L->hv_nseg, L->hv_seg, L->colval, X,
                                                                 partial);
            double* hp = part ? part + (size_t)grid * 2 * K : nullptr;
            const int32_t nh = L->hv_n;
            if (sub_mu)
                (stats ? k_heavy_final<T, LPR, true, true> : k_heavy_final<T, LPR, true, false>)
                    <<<kHeavyGrid, kBlock, 0, ctx->stream>>>(nh, L->hv_rows, L->hv_soff, partial, coef,
                                                             a_self, X, Y, mu, hp);
            else
                (stats ? k_heavy_final<T, LPR, false, true> : k_heavy_final<T, LPR, false, false>)
                    <<<kHeavyGrid, kBlock, 0, ctx->stream>>>(nh, L->hv_rows, L->hv_soff, partial, coef,
                                                             a_self, X, Y, mu, hp);
            sfg_toc(ctx);
            ctx->launches += 2;
            SFG_LAUNCH_CHECK(ctx, "heavy rows");
        }
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
        SFG_TRY(s.get(&part, (size_t)(grid + kHeavyGrid) * 2 * K));
        k_coef<<<sfg_grid(ctx, (const void*)k_coef, kBlock, 0, n), kBlock, 0, ctx->stream>>>(
            n, L->invdeg, omega, coef); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_coef");
        // ping-pong so that the last sweep writes `buf` and the projection writes X_out
        T* cur = (steps % 2 == 0) ? buf : X_out;
        T* nxt = (cur == buf) ? X_out : buf;
        sfg_tic(ctx, "init");
        if (steps == 0)
            k_init<T, LPR, false><<<grid, kBlock, 0, ctx->stream>>>(n, seed, L->deg, cur, part);
        else
            k_init<T, LPR, true><<<grid, kBlock, 0, ctx->stream>>>(n, seed, L->deg, cur, part);
        ++ctx->launches;
        sfg_toc(ctx);
        SFG_LAUNCH_CHECK(ctx, "k_init");
        k_finalize<<<K, kBlock, 0, ctx->stream>>>(part, grid, K, n, steps == 0 ? 1 : 2, mu, scale); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_finalize");
        for (int t = 1; t <= steps; ++t) {
            SFG_TRY(sweep(ctx, L, coef, (float)(1.0 - omega), cur, nxt, mu, part, t == 1,
                          t == steps, grid));
            std::swap(cur, nxt);
        }
        if (steps > 0) {
            k_finalize<<<K, kBlock, 0, ctx->stream>>>(part, part_slots(L, grid), K, n, 1, mu, scale); ++ctx->launches;
            SFG_LAUNCH_CHECK(ctx, "k_finalize");
        }
        sfg_tic(ctx, "project");
        k_project<T, LPR><<<sfg_grid(ctx, (const void*)k_project<T, LPR>, kBlock, 0,
                                     (int64_t)n * LPR),
                            kBlock, 0, ctx->stream>>>(n, cur, X_out, mu, scale); ++ctx->launches;
        sfg_toc(ctx);
        SFG_LAUNCH_CHECK(ctx, "k_project");
        return SFG_OK;
    }

    // Multicolour Gauss-Seidel smoothing: seeded block with its y-weighted column mean removed
    // (y: the weights of the quantity the ordered sweep conserves, so the block converges to
    // zero instead of to a constant; a constant shift commutes with the sweeps and the final
    // projection removes it either way), `steps` sweeps of one launch per colour class in
    // place, projection.
    static sfg_status smooth_gs(sfg_ctx* ctx, const sfg_graph* L, int steps, double omega,
                                uint64_t seed, T* X_out) {
        const int32_t n = L->n;
        SFG_TRY(sfg_gs_prepare(ctx, L));
        const int grid = grid_jacobi(ctx, n);
        const int gstat = sfg_grid(ctx, (const void*)k_col_stats<T, LPR>, kBlock, 0, (int64_t)n * LPR);
        Scratch s(ctx);
        T* buf;
        float *coef, *mu, *scale;
        double* part;
        SFG_TRY(s.get(&buf, (size_t)n * K));
        SFG_TRY(s.get(&coef, (size_t)n));
        SFG_TRY(s.get(&mu, K));
        SFG_TRY(s.get(&scale, K));
        SFG_TRY(s.get(&part, (size_t)std::max(grid, gstat) * 2 * K));
        double* yw;
        SFG_TRY(s.get(&yw, (size_t)n));
        k_coef<<<sfg_grid(ctx, (const void*)k_coef, kBlock, 0, n), kBlock, 0, ctx->stream>>>(
            n, L->invdeg, omega, coef);
        k_gs_weights<<<sfg_grid(ctx, (const void*)k_gs_weights, kBlock, 0, n), kBlock, 0,
                       ctx->stream>>>(n, L->row_ptr, L->colval, L->gs_color, omega, yw);
        if (L->hv_n > 0) {
            k_gs_weights_heavy<<<std::min(L->hv_n, 4 * ctx->num_sms), 256, 0, ctx->stream>>>(
                L->hv_n, L->hv_rows, L->row_ptr, L->colval, L->gs_color, omega, yw);
            ++ctx->launches;
        }
        k_init<T, LPR, true><<<grid, kBlock, 0, ctx->stream>>>(n, seed, yw, X_out, part);
        k_finalize<<<K, kBlock, 0, ctx->stream>>>(part, grid, K, n, 2, mu, scale);
        k_fill<<<1, 64, 0, ctx->stream>>>(K, 1.0f, scale);
        const int gp = sfg_grid(ctx, (const void*)k_project<T, LPR>, kBlock, 0, (int64_t)n * LPR);
        k_project<T, LPR><<<gp, kBlock, 0, ctx->stream>>>(n, X_out, buf, mu, scale);
        ctx->launches += 6;
        SFG_LAUNCH_CHECK(ctx, "gs init");
        const float a_self = (float)(1.0 - omega);
        const int ncol = (int)L->gs_off.size() - 1;
        SFG_TRY(gs_heavy_prepare(ctx, L));
        const int32_t hmax = L->hv_n > 0 ? kHeavy : INT32_MAX;
        int64_t max_seg = 0;
        for (int c = 0; c < ncol; ++c) max_seg = std::max(max_seg, L->gh_scoff[c + 1] - L->gh_scoff[c]);
        float* partial = nullptr;
        if (max_seg > 0) SFG_TRY(s.get(&partial, (size_t)max_seg * K));
        for (int t = 0; t < steps; ++t)
            for (int c = 0; c < ncol; ++c) {
                const int64_t c0 = L->gs_off[c], cnt = L->gs_off[c + 1] - c0;
                if (cnt == 0) continue;
                const int g = sfg_grid(ctx, (const void*)k_gs<T, LPR>, kBlock, 0, cnt * LPR);
                k_gs<T, LPR><<<g, kBlock, 0, ctx->stream>>>((int32_t)cnt, L->gs_order + c0,
                                                            L->row_ptr, L->colval, coef, a_self, buf,
                                                            hmax);
                ++ctx->launches;
                const int64_t nhc = L->gh_coff[c + 1] - L->gh_coff[c];
                if (nhc > 0) {  // this class's rows over the tile limit
                    const int64_t s0 = L->gh_scoff[c], nsc = L->gh_scoff[c + 1] - s0;
                    const int gp = sfg_grid(ctx, (const void*)k_heavy_part<T, LPR>, kBlock, 0, nsc * LPR);
                    k_heavy_part<T, LPR><<<gp, kBlock, 0, ctx->stream>>>(nsc, L->gh_seg + s0, L->colval,
                                                                         buf, partial);
                    const int gf = sfg_grid(ctx, (const void*)k_heavy_final_gs<T, LPR>, kBlock, 0,
                                            nhc * LPR);
                    k_heavy_final_gs<T, LPR><<<gf, kBlock, 0, ctx->stream>>>(
                        (int32_t)nhc, L->gh_rows + L->gh_coff[c], L->gh_soff + L->gh_coff[c], s0, partial,
                        coef, a_self, buf);
                    ctx->launches += 2;
                }
            }
        SFG_LAUNCH_CHECK(ctx, "k_gs");
        k_col_stats<T, LPR><<<gstat, kBlock, 0, ctx->stream>>>(n, buf, part);
        k_finalize<<<K, kBlock, 0, ctx->stream>>>(part, gstat, K, n, 1, mu, scale);
        k_project<T, LPR><<<gp, kBlock, 0, ctx->stream>>>(n, buf, X_out, mu, scale);
        ctx->launches += 3;
        SFG_LAUNCH_CHECK(ctx, "gs projection");
        return SFG_OK;
    }

    // Sweeps of one Laplacian from the block x0 (not overwritten) through the ping-pong pair
    // (b0, b1); *out = the raw smoothed block, mean/scale = its projection statistics.
    static sfg_status sweeps_from(sfg_ctx* ctx, const sfg_graph* L, int steps, double omega,
                                  int grid, const T* x0, T* b0, T* b1, const float* mu,
                                  double* part, float* coef, float* mean, float* scale,
                                  const T** out) {
        const int32_t n = L->n;
        k_coef<<<sfg_grid(ctx, (const void*)k_coef, kBlock, 0, n), kBlock, 0, ctx->stream>>>(
            n, L->invdeg, omega, coef);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_coef");
        const T* cur = x0;
        T* nxt = b0;
        for (int t = 1; t <= steps; ++t) {
            SFG_TRY(sweep(ctx, L, coef, (float)(1.0 - omega), cur, nxt, mu, part, t == 1,
                          t == steps, grid));
            cur = nxt;
            nxt = (nxt == b0) ? b1 : b0;
        }
        if (steps > 0) {
            k_finalize<<<K, kBlock, 0, ctx->stream>>>(part, part_slots(L, grid), K, n, 1, mean, scale);
            ++ctx->launches;
            SFG_LAUNCH_CHECK(ctx, "k_finalize");
        }
        *out = cur;
        return SFG_OK;
    }

    // Filter + score: one seeded block, swept on L_G and on L_P, scored with the projection
    // folded into the scorer (its mean removal cancels in X_p - X_q; its scaling is per column).
    static sfg_status filter_score(sfg_ctx* ctx, const sfg_graph* LG, const sfg_graph* LP,
                                   int steps, double omega, uint64_t seed, const int32_t* ids,
                                   int64_t ne, sfg_score_mode mode, float* scores) {
        const int32_t n = LG->n;
        const int grid = grid_jacobi(ctx, n);
        Scratch s(ctx);
        T *x0, *g0, *g1, *p0, *p1;
        float *coef, *mu, *mu_scale, *mg, *sg, *mp, *sp;
        double* part;
        SFG_TRY(s.get(&x0, (size_t)n * K));
        SFG_TRY(s.get(&g0, (size_t)n * K));
        SFG_TRY(s.get(&g1, (size_t)n * K));
        SFG_TRY(s.get(&p0, (size_t)n * K));
        SFG_TRY(s.get(&p1, (size_t)n * K));
        SFG_TRY(s.get(&coef, (size_t)n));
        SFG_TRY(s.get(&mu, K));
        SFG_TRY(s.get(&mu_scale, K));
        SFG_TRY(s.get(&mg, K));
        SFG_TRY(s.get(&sg, K));
        SFG_TRY(s.get(&mp, K));
        SFG_TRY(s.get(&sp, K));
        SFG_TRY(s.get(&part, (size_t)(grid + kHeavyGrid) * 2 * K));
        sfg_tic(ctx, "init");
        // the D-weighted mean is taken on L_G; L_P has the same nodes, and any constant left in
        // the block is removed by the projection in exact arithmetic
        if (steps == 0)
            k_init<T, LPR, false><<<grid, kBlock, 0, ctx->stream>>>(n, seed, LG->deg, x0, part);
        else
            k_init<T, LPR, true><<<grid, kBlock, 0, ctx->stream>>>(n, seed, LG->deg, x0, part);
        ++ctx->launches;
        sfg_toc(ctx);
        SFG_LAUNCH_CHECK(ctx, "k_init");
        // steps == 0: the projection statistics of both blocks are those of x0
        k_finalize<<<K, kBlock, 0, ctx->stream>>>(part, grid, K, n, steps == 0 ? 1 : 2, mu, mu_scale);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_finalize");
        const T *xg = x0, *xp = x0;
        SFG_TRY(sweeps_from(ctx, LG, steps, omega, grid, x0, g0, g1, mu, part, coef, mg, sg, &xg));
        SFG_TRY(sweeps_from(ctx, LP, steps, omega, grid, x0, p0, p1, mu, part, coef, mp, sp, &xp));
        if (steps == 0) sg = sp = mu_scale;
        return sfg_score_impl(ctx, LG, xg, xp, K, Vec<T>::E == 4 ? SFG_F32 : SFG_BF16, ids, ne,
                              mode, scores, sg, sp);
    }

    // Batched filter + score over a disjoint union (U, PU) of ng graphs (node_off on the device,
    // ng + 1 entries): per-graph seeded blocks, means and projection scales; one launch per sweep
    // for all graphs.
    static sfg_status filter_score_batched(sfg_ctx* ctx, const sfg_graph* U, const sfg_graph* PU,
                                           const int32_t* orig_local,
                                           int ng, const int32_t* node_off, int steps,
                                           double omega, uint64_t seed, const int32_t* ids,
                                           int64_t ne, sfg_score_mode mode, float* scores) {
        const int32_t n = U->n;
        const int grid = grid_jacobi(ctx, n);
        Scratch s(ctx);
        T *x0, *g0, *g1, *p0, *p1;
        float *coef, *mean, *sg, *sp;
        double* stats;
        SFG_TRY(s.get(&x0, (size_t)n * K));
        SFG_TRY(s.get(&g0, (size_t)n * K));
        SFG_TRY(s.get(&g1, (size_t)n * K));
        SFG_TRY(s.get(&p0, (size_t)n * K));
        SFG_TRY(s.get(&p1, (size_t)n * K));
        SFG_TRY(s.get(&coef, (size_t)n));
        SFG_TRY(s.get(&mean, (size_t)ng * K));
        SFG_TRY(s.get(&sg, (size_t)ng * K));
        SFG_TRY(s.get(&sp, (size_t)ng * K));
        SFG_TRY(s.get(&stats, (size_t)ng * 2 * K));
        double* spart;
        SFG_TRY(s.get(&spart, (size_t)ng * kSegSlices * 2 * K));
        const unsigned fin_grid = ceil_div_u((int64_t)ng * K, kBlock);
        const unsigned red_grid = ceil_div_u((int64_t)ng * 2 * K, kBlock);
        auto seg_stats = [&](const T* X, const double* deg) {
            k_seg_stats<T, LPR><<<ng * kSegSlices, kBlock, 0, ctx->stream>>>(X, node_off, deg, spart);
            k_seg_reduce<<<red_grid, kBlock, 0, ctx->stream>>>(ng, 2 * K, spart, stats);
            ctx->launches += 2;
        };
        k_init_batched<T, LPR><<<grid, kBlock, 0, ctx->stream>>>(n, seed, node_off, ng, orig_local, x0);
        const bool weighted = steps > 0;
        seg_stats(x0, weighted ? U->deg : nullptr);
        k_seg_finalize<<<fin_grid, kBlock, 0, ctx->stream>>>(stats, node_off, ng, K, weighted ? 1 : 0,
                                                             mean, nullptr);
        k_center_batched<T, LPR><<<grid, kBlock, 0, ctx->stream>>>(n, node_off, ng, mean, x0);
        ctx->launches += 3;
        SFG_LAUNCH_CHECK(ctx, "k_init_batched");
        const T* xr[2] = {x0, x0};
        const sfg_graph* L[2] = {U, PU};
        T* buf[2][2] = {{g0, g1}, {p0, p1}};
        float* sc[2] = {sg, sp};
        for (int w = 0; w < 2; ++w) {
            k_coef<<<sfg_grid(ctx, (const void*)k_coef, kBlock, 0, n), kBlock, 0, ctx->stream>>>(
                n, L[w]->invdeg, omega, coef);
            ++ctx->launches;
            SFG_LAUNCH_CHECK(ctx, "k_coef");
            const T* cur = x0;
            T* nxt = buf[w][0];
            for (int t = 1; t <= steps; ++t) {
                SFG_TRY(sweep(ctx, L[w], coef, (float)(1.0 - omega), cur, nxt, nullptr, nullptr,
                              false, false, grid));
                cur = nxt;
                nxt = (nxt == buf[w][0]) ? buf[w][1] : buf[w][0];
            }
            xr[w] = cur;
            seg_stats(cur, nullptr);
            k_seg_finalize<<<fin_grid, kBlock, 0, ctx->stream>>>(stats, node_off, ng, K, 0, mean, sc[w]);
            ++ctx->launches;
            SFG_LAUNCH_CHECK(ctx, "k_seg_stats");
        }
        return sfg_score_batched_impl(ctx, U, xr[0], xr[1], K, Vec<T>::E == 4 ? SFG_F32 : SFG_BF16,
                                      ids, ne, mode, scores, sg, sp, node_off, ng);
    }

    // Time every tile-shape variant of the plain sweep on L and record the fastest.
    static sfg_status autotune(sfg_ctx* ctx, const sfg_graph* L, int* best_host, double* us_host) {
        const int32_t n = L->n;
        const int grid = grid_jacobi(ctx, n);
        Scratch s(ctx);
        T *x, *y;
        float* coef;
        double* part;
        SFG_TRY(s.get(&x, (size_t)n * K));
        SFG_TRY(s.get(&y, (size_t)n * K));
        SFG_TRY(s.get(&coef, (size_t)n));
        SFG_TRY(s.get(&part, (size_t)(grid + kHeavyGrid) * 2 * K));
        k_init<T, LPR, false><<<grid, kBlock, 0, ctx->stream>>>(n, 12345, L->deg, x, part);
        k_coef<<<sfg_grid(ctx, (const void*)k_coef, kBlock, 0, n), kBlock, 0, ctx->stream>>>(
            n, L->invdeg, 0.7, coef);
        ctx->launches += 2;
        SFG_LAUNCH_CHECK(ctx, "autotune init");
        cudaEvent_t e0, e1;
        SFG_CUDA(ctx, cudaEventCreate(&e0));
        SFG_CUDA(ctx, cudaEventCreate(&e1));
        SFG_TRY(heavy_prepare(ctx, L));  // the tile kernel is timed as the sweep runs it
        const int32_t hmax = L->hv_n > 0 ? kHeavy : INT32_MAX;
        int best = kJDefault;
        float best_ms = 1e30f;
        const float a_self = 0.3f;
        const float* mu = nullptr;
        double* pp = nullptr;
        for (int v = 0; v < kJNumVariants; ++v) {
            void* k = plain_kern(v);
            const int g = sfg_grid(ctx, k, kBlock, 0, (int64_t)n * LPR);
            const T* X = x;
            T* Y = y;
            void* args[] = {(void*)&n, (void*)&hmax, (void*)&L->row_ptr, (void*)&L->colval, (void*)&coef,
                            (void*)&a_self, (void*)&X, (void*)&Y, (void*)&mu, (void*)&pp};
            for (int r = 0; r < 4; ++r) {  // one warm-up, three timed
                if (r == 1) cudaEventRecord(e0, ctx->stream);
                const cudaError_t err = cudaLaunchKernel(k, dim3(g), dim3(kBlock), args, 0, ctx->stream);
                ++ctx->launches;
                if (err != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return sfg_cuda_fail(ctx, err, "autotune sweep");
                }
            }
            cudaEventRecord(e1, ctx->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) { best_ms = ms; best = v; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        sfg_tune_record(ctx, K, Vec<T>::E == 4 ? SFG_F32 : SFG_BF16, L, best);
        SFG_TRY(sfg_score_autotune_impl(ctx, L, K, Vec<T>::E == 4 ? SFG_F32 : SFG_BF16, x));
        if (best_host) *best_host = best;
        if (us_host) *us_host = best_ms / 3.0 * 1e3;
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
            n, L->invdeg, omega, coef); ++ctx->launches;
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

sfg_status sfg_heavy_prepare(sfg_ctx* ctx, const sfg_graph* L) { return heavy_prepare(ctx, L); }

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

sfg_status sfg_smooth_gs_impl(sfg_ctx* ctx, const sfg_graph* L, int K, int steps, double omega,
                              uint64_t seed, sfg_dtype storage, void* X_out) {
    return dispatch(K, storage, [&](auto S) {
        using Sm = decltype(S);
        return Sm::smooth_gs(ctx, L, steps, omega, seed, static_cast<typename Sm::Elem*>(X_out));
    });
}

sfg_status sfg_filter_score_impl(sfg_ctx* ctx, const sfg_graph* LG, const sfg_graph* LP, int K,
                                 int steps, double omega, uint64_t seed, sfg_dtype storage,
                                 const int32_t* ids, int64_t ne, sfg_score_mode mode,
                                 float* scores) {
    return dispatch(K, storage, [&](auto S) {
        using Sm = decltype(S);
        return Sm::filter_score(ctx, LG, LP, steps, omega, seed, ids, ne, mode, scores);
    });
}

sfg_status sfg_filter_score_batched_impl(sfg_ctx* ctx, const sfg_graph* U, const sfg_graph* PU,
                                         const int32_t* orig_local,
                                         int ng, const int32_t* node_off, int K, int steps,
                                         double omega, uint64_t seed, sfg_dtype storage,
                                         const int32_t* ids, int64_t ne, sfg_score_mode mode,
                                         float* scores) {
    return dispatch(K, storage, [&](auto S) {
        using Sm = decltype(S);
        return Sm::filter_score_batched(ctx, U, PU, orig_local, ng, node_off, steps, omega, seed,
                                        ids, ne, mode, scores);
    });
}

sfg_status sfg_autotune_impl(sfg_ctx* ctx, const sfg_graph* L, int K, sfg_dtype storage,
                             int* best, double* us) {
    return dispatch(K, storage, [&](auto S) {
        using Sm = decltype(S);
        return Sm::autotune(ctx, L, best, us);
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
    SFG_DEVICE(ctx);
    SFG_TRY(check_smooth_args(ctx, L, K, steps, omega, storage, X_out));
    return sfg_smooth_impl(ctx, L, K, steps, omega, seed, storage, X_out);
}

sfg_status sfg_smooth_gs(sfg_ctx* ctx, const sfg_graph* L, int K, int steps, double omega,
                         uint64_t seed, sfg_dtype storage, void* X_out) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!(omega > 0.0 && omega < 2.0))
        return sfg_fail(ctx, SFG_EINVAL, "omega must be in (0, 2) for Gauss-Seidel");
    SFG_TRY(check_smooth_args(ctx, L, K, steps, 1.0, storage, X_out));
    return sfg_smooth_gs_impl(ctx, L, K, steps, omega, seed, storage, X_out);
}

sfg_status sfg_jacobi(sfg_ctx* ctx, const sfg_graph* L, int K, int steps, double omega,
                      sfg_dtype storage, void* X_inout) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    SFG_TRY(check_smooth_args(ctx, L, K, steps, omega, storage, X_inout));
    return dispatch(K, storage, [&](auto S) {
        using Sm = decltype(S);
        return Sm::jacobi(ctx, L, steps, omega, static_cast<typename Sm::Elem*>(X_inout));
    });
}

sfg_status sfg_filter_score(sfg_ctx* ctx, const sfg_graph* LG, const sfg_graph* LP, int K,
                            int steps, double omega, uint64_t seed, sfg_dtype storage,
                            const int32_t* edge_ids, int64_t ne, sfg_score_mode mode,
                            float* scores_out) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!LG || !LP) return sfg_fail(ctx, SFG_EINVAL, "graph is NULL");
    if (LG->n != LP->n) return sfg_fail(ctx, SFG_EINVAL, "L_G and L_P differ in node count");
    if (!sfg_k_supported(K, storage))
        return sfg_fail(ctx, SFG_EUNSUPPORTED, "K=%d unsupported for dtype %d", K, (int)storage);
    if (steps < 0) return sfg_fail(ctx, SFG_EINVAL, "steps must be >= 0");
    if (!(omega > 0.0 && omega <= 1.0)) return sfg_fail(ctx, SFG_EINVAL, "omega must be in (0, 1]");
    if (ne < 0) return sfg_fail(ctx, SFG_EINVAL, "ne must be >= 0");
    if (mode != SFG_SCORE_RATIO && mode != SFG_SCORE_G && mode != SFG_SCORE_P)
        return sfg_fail(ctx, SFG_EINVAL, "unknown score mode %d", (int)mode);
    if (ne == 0) return SFG_OK;
    SFG_TRY(sfg_check_dev(ctx, edge_ids, "edge_ids"));
    SFG_TRY(sfg_check_dev(ctx, scores_out, "scores_out"));
    return sfg_filter_score_impl(ctx, LG, LP, K, steps, omega, seed, storage, edge_ids, ne, mode,
                                 scores_out);
}

}  // extern "C"
