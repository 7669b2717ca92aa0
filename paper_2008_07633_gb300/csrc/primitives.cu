// Device-wide primitives: exclusive scan and a stable LSD radix sort of (uint64 key, uint32 value)
// pairs. Both are plain three-phase designs (per-tile reduce, scan of tile totals, per-tile apply)
// that keep every pass a coalesced sweep over HBM.
#include "sfg_internal.cuh"

namespace {

constexpr int kScanBlock = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;

// Exclusive scan of one value per thread over a 256-thread block; returns the block total.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
    __shared__ int64_t warp_tot[kScanBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < kScanBlock / 32 ? warp_tot[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kScanBlock / 32) warp_tot[lane] = wi - w;  // exclusive warp offsets
        if (lane == kScanBlock / 32 - 1) *total = wi;
    }
    __syncthreads();
    int64_t r = warp_tot[warp] + inc - v;
    __syncthreads();
    return r;
}

template <typename T>
__global__ void k_scan_reduce(const T* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + (int64_t)i * kScanBlock + threadIdx.x;
        if (idx < n) s += (int64_t)in[idx];
    }
    __shared__ int64_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// The tile's results pass through shared memory (one padding slot per 16 entries keeps the
// thread-ordered writes free of bank conflicts), so that the global stores are coalesced.
__device__ __forceinline__ int scan_slot(int p) { return p + (p >> 4); }

template <typename T>
__global__ void k_scan_apply(const T* __restrict__ in, int64_t n, const int64_t* __restrict__ offs,
                             int64_t nb, int64_t* __restrict__ out) {
    __shared__ int64_t so[kScanTile + kScanTile / 16];
    const int64_t tile0 = (int64_t)blockIdx.x * kScanTile;
    const int64_t base = tile0 + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? (int64_t)in[idx] : 0;
        s += v[i];
    }
    __shared__ int64_t tot;
    int64_t run = block_exclusive_scan(s, &tot) + offs[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        so[scan_slot(threadIdx.x * kScanItems + i)] = run;
        run += v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int q = i * kScanBlock + threadIdx.x;
        if (tile0 + q < n) out[tile0 + q] = so[scan_slot(q)];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = offs[nb];
}

// Single-tile scan used when everything fits one block: writes out[0..n] directly.
template <typename T>
__global__ void k_scan_single(const T* __restrict__ in, int64_t n, int64_t* __restrict__ out) {
    const int64_t base = (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? (int64_t)in[idx] : 0;
        s += v[i];
    }
    __shared__ int64_t tot;
    int64_t run = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (threadIdx.x == 0) out[n] = tot;
}

template <typename T>
sfg_status scan_impl(sfg_ctx* ctx, const T* in, int64_t* out, int64_t n) {
    if (n <= kScanTile) {
        k_scan_single<T><<<1, kScanBlock, 0, ctx->stream>>>(in, n, out); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_scan_single");
        return SFG_OK;
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    Scratch s(ctx);
    int64_t *sums, *offs;
    SFG_TRY(s.get(&sums, nb));
    SFG_TRY(s.get(&offs, nb + 1));
    k_scan_reduce<T><<<(unsigned)nb, kScanBlock, 0, ctx->stream>>>(in, n, sums); ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_scan_reduce");
    SFG_TRY(scan_impl<int64_t>(ctx, sums, offs, nb));
    k_scan_apply<T><<<(unsigned)nb, kScanBlock, 0, ctx->stream>>>(in, n, offs, nb, out); ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_scan_apply");
    return SFG_OK;
}

// ------------------------------------------------------------------------------------------------
// Radix sort: 8-bit digits, tiles of 2048 pairs per 256-thread block (8 warps x 8 rounds of 32;
// 64 registers, four CTAs per SM: 15% faster than 4096-pair tiles at two CTAs per SM).
// Pass = histogram per tile -> exclusive scan of the digit-major count table -> stable scatter.
// Stability inside a tile comes from ranking each round's 32 items with __match_any_sync and
// accumulating per-warp digit counters in order; warps are then offset by an exclusive scan
// over warps, so the tile keeps input order among equal digits. The scatter first reorders the
// tile by digit in shared memory and then writes it out in that order, so each digit's run of
// the tile (8 pairs on average) leaves as consecutive stores instead of one store per pair.
// ------------------------------------------------------------------------------------------------
constexpr int kSortBlock = 256;
constexpr int kSortRounds = 8;
constexpr int kSortWarps = kSortBlock / 32;
constexpr int kSortTile = kSortBlock * kSortRounds;
constexpr int kRadix = 256;

__global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int64_t nb,
                             int32_t* __restrict__ counts) {
    __shared__ int32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = 0; i < kSortRounds; ++i) {
        int64_t idx = base + (int64_t)i * kSortBlock + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 0xff], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];  // digit-major
}

constexpr size_t kScatterSmem = (size_t)kSortTile * (sizeof(uint64_t) + sizeof(uint32_t));

__global__ void __launch_bounds__(kSortBlock)
    k_radix_scatter(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                    int64_t n, int shift, int64_t nb, const int64_t* __restrict__ offs,
                    uint64_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out) {
    __shared__ int32_t wcnt[kSortWarps][kRadix];
    __shared__ int64_t gbase[kRadix];
    __shared__ int32_t tstart[kRadix];  // first tile-local position of each digit
    extern __shared__ __align__(16) unsigned char s_tile[];
    uint64_t* sk = reinterpret_cast<uint64_t*>(s_tile);
    uint32_t* sv = reinterpret_cast<uint32_t*>(sk + kSortTile);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kSortWarps * kRadix; d += kSortBlock) (&wcnt[0][0])[d] = 0;
    gbase[threadIdx.x] = offs[(int64_t)threadIdx.x * nb + blockIdx.x];
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * (32 * kSortRounds);
    const unsigned lt = (1u << lane) - 1u;
    uint64_t k[kSortRounds];
    uint32_t v[kSortRounds];
    int32_t rank[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t idx = base + r * 32 + lane;
        const bool ok = idx < n;
        k[r] = ok ? keys[idx] : 0;
        v[r] = ok ? vals[idx] : 0;
        const int d = ok ? (int)((k[r] >> shift) & 0xff) : kRadix;  // out-of-range lanes match apart
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int before = __popc(peers & lt);
        const int32_t cur = wcnt[warp][ok ? d : 0];
        rank[r] = ok ? cur + before : 0;
        __syncwarp();
        if (ok && before == 0) wcnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // exclusive scan over warps, per digit; the digit's total is its tile count
        const int d = threadIdx.x;
        int32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            int32_t t = wcnt[w][d];
            wcnt[w][d] = run;
            run += t;
        }
        tstart[d] = run;
    }
    __syncthreads();
    {   // exclusive scan of the tile's digit counts over digits (one digit per thread)
        __shared__ int32_t wsum[kSortWarps];
        const int32_t c = tstart[threadIdx.x];
        int32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t q = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += q;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        int32_t before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        tstart[threadIdx.x] = before + inc - c;
    }
    __syncthreads();
    // the tile in digit order in shared memory (stable: equal digits keep input order)
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t idx = base + r * 32 + lane;
        if (idx < n) {
            const int d = (int)((k[r] >> shift) & 0xff);
            const int32_t lp = tstart[d] + wcnt[warp][d] + rank[r];
            sk[lp] = k[r];
            sv[lp] = v[r];
        }
    }
    __syncthreads();
    // out in that order: position i of the tile goes to its digit's global run
    const int64_t left = n - (int64_t)blockIdx.x * kSortTile;
    const int32_t cnt = left < kSortTile ? (int32_t)left : kSortTile;
    for (int32_t i = threadIdx.x; i < cnt; i += kSortBlock) {
        const uint64_t key = sk[i];
        const int d = (int)((key >> shift) & 0xff);
        const int64_t pos = gbase[d] + (i - tstart[d]);
        keys_out[pos] = key;
        vals_out[pos] = sv[i];
    }
}

}  // namespace

sfg_status sfg_scan_u8(sfg_ctx* ctx, const uint8_t* in, int64_t* out, int64_t n) {
    return scan_impl<uint8_t>(ctx, in, out, n);
}
sfg_status sfg_scan_i32(sfg_ctx* ctx, const int32_t* in, int64_t* out, int64_t n) {
    return scan_impl<int32_t>(ctx, in, out, n);
}
sfg_status sfg_scan_i64(sfg_ctx* ctx, const int64_t* in, int64_t* out, int64_t n) {
    return scan_impl<int64_t>(ctx, in, out, n);
}

sfg_status sfg_radix_sort_pairs(sfg_ctx* ctx, uint64_t** keys, uint32_t** vals,
                                uint64_t** keys_alt, uint32_t** vals_alt, int64_t n, int bits) {
    if (n <= 1 || bits <= 0) return SFG_OK;
    const int64_t nb = (n + kSortTile - 1) / kSortTile;
    Scratch s(ctx);
    int32_t* counts;
    int64_t* offs;
    SFG_TRY(s.get(&counts, (size_t)kRadix * nb));
    SFG_TRY(s.get(&offs, (size_t)kRadix * nb + 1));
    {   // the scatter's tile buffer is above the default shared-memory limit: opt in once
        const auto key = std::make_tuple((const void*)k_radix_scatter, kSortBlock, kScatterSmem);
        if (ctx->occupancy.find(key) == ctx->occupancy.end()) {
            SFG_CUDA(ctx, cudaFuncSetAttribute(k_radix_scatter,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kScatterSmem));
            ctx->occupancy.emplace(key, 0);
        }
    }
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)nb, kSortBlock, 0, ctx->stream>>>(*keys, n, shift, nb, counts); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_radix_hist");
        SFG_TRY(sfg_scan_i32(ctx, counts, offs, (int64_t)kRadix * nb));
        k_radix_scatter<<<(unsigned)nb, kSortBlock, kScatterSmem, ctx->stream>>>(
            *keys, *vals, n, shift, nb, offs, *keys_alt, *vals_alt); ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_radix_scatter");
        std::swap(*keys, *keys_alt);
        std::swap(*vals, *vals_alt);
    }
    return SFG_OK;
}

sfg_status sfg_read_i64(sfg_ctx* ctx, const int64_t* dev, int64_t* host) {
    SFG_CUDA(ctx, cudaMemcpyAsync(host, dev, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SFG_OK;
}
