// Top-k selection (the selection step of Algorithm 1: the candidate edges of largest distortion
// are added to the sparsifier).
//
// Each candidate becomes a unique 64-bit key: the order-preserving image of its FP32 score in the
// high word and the complement of its id in the low word, so "larger key" is exactly the strict
// order (score descending, id ascending). An MSB-first radix select (8 passes of 8-bit digits,
// histogram in shared memory, the digit pick done on the device) finds the k-th largest key
// without any host round trip; one compaction pass keeps the keys at or above it and a small
// radix sort returns the chosen ids in ascending order.
#include "sfg_internal.cuh"

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ uint64_t sel_key(float s, int32_t id) {
    const uint32_t b = __float_as_uint(s);
    const uint32_t o = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return ((uint64_t)o << 32) | (uint64_t)(~(uint32_t)id);
}

struct SelState {
    unsigned long long prefix;
    long long krem;
    unsigned long long hist[256];
};

__global__ void k_sel_init(SelState* st, int64_t k) {
    st->prefix = 0ull;
    st->krem = k;
    for (int d = threadIdx.x; d < 256; d += blockDim.x) st->hist[d] = 0ull;
}

__global__ void __launch_bounds__(kBlock)
    k_sel_hist(int64_t ne, const float* __restrict__ scores, const int32_t* __restrict__ ids,
               int shift, SelState* __restrict__ st) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t prefix = st->prefix;
    const int hi = shift + 8;  // bits at and above `hi` must match the prefix
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < ne;
         i += (int64_t)gridDim.x * kBlock) {
        const uint64_t key = sel_key(scores[i], ids[i]);
        if (hi >= 64 || (key >> hi) == (prefix >> hi)) atomicAdd(&h[(key >> shift) & 0xff], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&st->hist[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

// Pick the digit holding the k-th largest key: suffix sums over the 256 buckets by a block scan
// (thread d holds bucket 255 - d), then the first bucket whose suffix reaches krem.
__global__ void k_sel_pick(int shift, SelState* st) {
    __shared__ long long suf[256];
    const int d = 255 - (int)threadIdx.x;
    const long long c = (long long)st->hist[d];
    suf[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {  // inclusive scan from the top bucket down
        const long long v = threadIdx.x >= o ? suf[threadIdx.x - o] : 0;
        __syncthreads();
        suf[threadIdx.x] += v;
        __syncthreads();
    }
    const long long krem = st->krem;
    const long long incl = suf[threadIdx.x], above = incl - c;
    const bool pick = (above < krem && incl >= krem) || (d == 0 && incl < krem);
    __syncthreads();
    if (pick) {
        st->prefix |= (unsigned long long)d << shift;
        st->krem = krem - above;
    }
    st->hist[d] = 0ull;
}

__global__ void k_sel_flags(int64_t ne, const float* __restrict__ scores,
                            const int32_t* __restrict__ ids, const SelState* __restrict__ st,
                            uint8_t* __restrict__ flag) {
    const uint64_t thr = st->prefix;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < ne;
         i += (int64_t)gridDim.x * kBlock)
        flag[i] = sel_key(scores[i], ids[i]) >= thr;
}

__global__ void k_sel_compact(int64_t ne, const int32_t* __restrict__ ids,
                              const uint8_t* __restrict__ flag, const int64_t* __restrict__ pos,
                              uint64_t* __restrict__ out_keys, uint32_t* __restrict__ out_vals) {
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < ne;
         i += (int64_t)gridDim.x * kBlock)
        if (flag[i]) {
            out_keys[pos[i]] = (uint64_t)(uint32_t)ids[i];
            out_vals[pos[i]] = 0u;
        }
}

__global__ void k_sel_emit(int64_t k, const uint64_t* __restrict__ keys, int32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < k;
         i += (int64_t)gridDim.x * kBlock)
        out[i] = (int32_t)keys[i];
}

}  // namespace

sfg_status sfg_topk_impl(sfg_ctx* ctx, const float* scores, const int32_t* ids, int64_t ne,
                         int64_t k, int32_t* out) {
    if (k == 0) return SFG_OK;
    Scratch s(ctx);
    SelState* st;
    uint8_t* flag;
    int64_t* pos;
    uint64_t *ka, *kb;
    uint32_t *va, *vb;
    SFG_TRY(s.get(&st, 1));
    SFG_TRY(s.get(&flag, ne));
    SFG_TRY(s.get(&pos, ne + 1));
    SFG_TRY(s.get(&ka, k));
    SFG_TRY(s.get(&kb, k));
    SFG_TRY(s.get(&va, k));
    SFG_TRY(s.get(&vb, k));
    const int grid = sfg_grid(ctx, (const void*)k_sel_hist, kBlock, 0, ne);
    sfg_tic(ctx, "topk");
    k_sel_init<<<1, kBlock, 0, ctx->stream>>>(st, k); ++ctx->launches;
    for (int shift = 56; shift >= 0; shift -= 8) {
        k_sel_hist<<<grid, kBlock, 0, ctx->stream>>>(ne, scores, ids, shift, st); ++ctx->launches;
        k_sel_pick<<<1, 256, 0, ctx->stream>>>(shift, st); ++ctx->launches;
    }
    k_sel_flags<<<grid, kBlock, 0, ctx->stream>>>(ne, scores, ids, st, flag); ++ctx->launches;
    sfg_toc(ctx);
    SFG_LAUNCH_CHECK(ctx, "k_sel");
    SFG_TRY(sfg_scan_u8(ctx, flag, pos, ne));
    k_sel_compact<<<grid, kBlock, 0, ctx->stream>>>(ne, ids, flag, pos, ka, va); ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_sel_compact");
    SFG_TRY(sfg_radix_sort_pairs(ctx, &ka, &va, &kb, &vb, k, 32));
    k_sel_emit<<<sfg_grid(ctx, (const void*)k_sel_emit, kBlock, 0, k), kBlock, 0, ctx->stream>>>(
        k, ka, out); ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_sel_emit");
    return SFG_OK;
}

extern "C" sfg_status sfg_select_topk(sfg_ctx* ctx, const float* scores, const int32_t* ids,
                                      int64_t ne, int64_t k, int32_t* ids_out) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (ne < 0 || k < 0 || k > ne)
        return sfg_fail(ctx, SFG_EINVAL, "need 0 <= k <= ne (k=%lld, ne=%lld)", (long long)k,
                        (long long)ne);
    if (k == 0) return SFG_OK;
    SFG_TRY(sfg_check_dev(ctx, scores, "scores"));
    SFG_TRY(sfg_check_dev(ctx, ids, "ids"));
    SFG_TRY(sfg_check_dev(ctx, ids_out, "ids_out"));
    return sfg_topk_impl(ctx, scores, ids, ne, k, ids_out);
}

// ------------------------------------------------------------------------------------------------
// Segmented top-k (one selection per graph of a batch): the same MSB-first radix select, with one
// histogram and one (prefix, remaining k) state per segment. Candidates are contiguous per
// segment; each warp sweeps one contiguous range of them, 32 at a time, so its segment (found once
// by a binary search) advances by a few steps at most and its state stays in registers.
// ------------------------------------------------------------------------------------------------
namespace {

struct SegSel {
    unsigned long long prefix;
    long long krem;
};

__device__ __forceinline__ int seg_of(const int64_t* __restrict__ off, int nseg, int64_t i) {
    int lo = 0, hi = nseg;  // last s with off[s] <= i
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_segsel_init(int nseg, const int64_t* __restrict__ k, SegSel* __restrict__ st,
                              unsigned long long* __restrict__ hist) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)nseg * 256;
         i += (int64_t)gridDim.x * blockDim.x) {
        hist[i] = 0ull;
        if ((i & 255) == 0) st[i >> 8] = SegSel{0ull, (long long)k[i >> 8]};
    }
}

// The contiguous item range [lo, hi) of this warp: ne split into equal chunks of whole 32-item steps.
__device__ __forceinline__ void warp_range(int64_t ne, int64_t& lo, int64_t& hi) {
    const int64_t nw = (int64_t)gridDim.x * (kBlock / 32);
    const int64_t w = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int64_t steps = (ne + 31) / 32, per = (steps + nw - 1) / nw;
    lo = min(ne, w * per * 32);
    hi = min(ne, (w + 1) * per * 32);
}

__global__ void __launch_bounds__(kBlock)
    k_segsel_hist(int64_t ne, const float* __restrict__ scores, const int32_t* __restrict__ ids,
                  int nseg, const int64_t* __restrict__ off, const SegSel* __restrict__ st,
                  int shift, unsigned long long* __restrict__ hist) {
    const int hi = shift + 8;
    int64_t lo_i, hi_i;
    warp_range(ne, lo_i, hi_i);
    if (lo_i >= hi_i) return;
    int s = seg_of(off, nseg, lo_i);  // this lane's segment, advanced as the range moves on
    int64_t s_end = off[s + 1];
    SegSel ss = st[s];
    for (int64_t base = lo_i; base < hi_i; base += 32) {
        const int64_t i = base + (threadIdx.x & 31);
        bool take = false;
        int digit = 0;
        if (i < hi_i) {
            if (i >= s_end) {
                do ++s; while (off[s + 1] <= i);
                s_end = off[s + 1];
                ss = st[s];
            }
            const uint64_t key = sel_key(scores[i], ids[i]);
            take = ss.krem > 0 && (hi >= 64 || (key >> hi) == (ss.prefix >> hi));
            digit = (int)((key >> shift) & 0xff);
        }
        const unsigned bin = take ? (unsigned)s * 256u + (unsigned)digit : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        if (take && (__ffs(peers) - 1) == (int)(threadIdx.x & 31))
            atomicAdd(&hist[bin], (unsigned long long)__popc(peers));
    }
}

// one CTA of 256 threads per segment (see k_sel_pick)
__global__ void k_segsel_pick(int shift, SegSel* __restrict__ st, unsigned long long* __restrict__ hist) {
    __shared__ long long suf[256];
    const int sgi = blockIdx.x;
    unsigned long long* h = hist + (size_t)sgi * 256;
    const long long krem = st[sgi].krem;
    const int d = 255 - (int)threadIdx.x;
    const long long c = (long long)h[d];
    suf[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        const long long v = threadIdx.x >= o ? suf[threadIdx.x - o] : 0;
        __syncthreads();
        suf[threadIdx.x] += v;
        __syncthreads();
    }
    const long long incl = suf[threadIdx.x], above = incl - c;
    const bool pick = krem > 0 && ((above < krem && incl >= krem) || (d == 0 && incl < krem));
    __syncthreads();
    if (pick) {
        st[sgi].prefix |= (unsigned long long)d << shift;
        st[sgi].krem = krem - above;
    }
    h[d] = 0ull;
}

__global__ void __launch_bounds__(kBlock)
    k_segsel_flags(int64_t ne, const float* __restrict__ scores, const int32_t* __restrict__ ids,
                   int nseg, const int64_t* __restrict__ off, const SegSel* __restrict__ st,
                   const int64_t* __restrict__ k, uint8_t* __restrict__ flag) {
    int64_t lo_i, hi_i;
    warp_range(ne, lo_i, hi_i);
    if (lo_i >= hi_i) return;
    int s = seg_of(off, nseg, lo_i);
    int64_t s_end = off[s + 1];
    bool on = k[s] > 0;
    uint64_t thr = st[s].prefix;
    for (int64_t i = lo_i + (threadIdx.x & 31); i < hi_i; i += 32) {
        if (i >= s_end) {
            do ++s; while (off[s + 1] <= i);
            s_end = off[s + 1];
            on = k[s] > 0;
            thr = st[s].prefix;
        }
        flag[i] = on && sel_key(scores[i], ids[i]) >= thr;
    }
}

__global__ void k_segsel_emit(int64_t ne, const int32_t* __restrict__ ids,
                              const uint8_t* __restrict__ flag, const int64_t* __restrict__ pos,
                              int32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < ne;
         i += (int64_t)gridDim.x * kBlock)
        if (flag[i]) out[pos[i]] = ids[i];
}

}  // namespace

sfg_status sfg_topk_segmented_impl(sfg_ctx* ctx, const float* scores, const int32_t* ids,
                                   int64_t ne, int nseg, const int64_t* seg_off,
                                   const int64_t* k_dev, int64_t k_total, int32_t* out) {
    if (k_total == 0 || ne == 0) return SFG_OK;
    Scratch s(ctx);
    SegSel* st;
    unsigned long long* hist;
    uint8_t* flag;
    int64_t* pos;
    SFG_TRY(s.get(&st, nseg));
    SFG_TRY(s.get(&hist, (size_t)nseg * 256));
    SFG_TRY(s.get(&flag, ne));
    SFG_TRY(s.get(&pos, ne + 1));
    const int grid = sfg_grid(ctx, (const void*)k_segsel_hist, kBlock, 0, ne);
    sfg_tic(ctx, "topk");
    k_segsel_init<<<ceil_div_u((int64_t)nseg * 256, kBlock), kBlock, 0, ctx->stream>>>(nseg, k_dev, st, hist);
    ++ctx->launches;
    for (int shift = 56; shift >= 0; shift -= 8) {
        k_segsel_hist<<<grid, kBlock, 0, ctx->stream>>>(ne, scores, ids, nseg, seg_off, st, shift, hist);
        k_segsel_pick<<<nseg, 256, 0, ctx->stream>>>(shift, st, hist);
        ctx->launches += 2;
    }
    k_segsel_flags<<<grid, kBlock, 0, ctx->stream>>>(ne, scores, ids, nseg, seg_off, st, k_dev, flag);
    ++ctx->launches;
    sfg_toc(ctx);
    SFG_LAUNCH_CHECK(ctx, "k_segsel");
    SFG_TRY(sfg_scan_u8(ctx, flag, pos, ne));
    k_segsel_emit<<<grid, kBlock, 0, ctx->stream>>>(ne, ids, flag, pos, out);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_segsel_emit");
    return SFG_OK;
}
