// Learned edge-proposal scorer (an addition to the paper's method; the proposals it makes are
// rescored by the plain method before selection): per-edge features from a short embedding, a 16 -> 64 -> 64 -> 1 ReLU network evaluated
// on the tcgen05 tensor cores (inference, k_mlp_forward_tc below) and trained on BF16 warp-level
// tensor-core MMA (mma.sync m16n8k16, FP32 accumulation), Adam in FP32.
//
// Training forward, per warp and 16 edges: the feature rows are the A operand; layer outputs stay in the
// accumulator fragments, whose layout is exactly the A-operand layout of the next layer once two
// n-tiles are packed to BF16, so hidden activations never leave registers. The last layer (64 -> 1)
// is a dot product folded across the four lanes that share a row.
// Backward, per CTA (4 warps, 64 edges): delta_1 = delta_2 W2^T reuses the same register trick
// with a fragment copy of W2^T; the weight gradients H1^T delta_2 and X^T delta_1 contract over
// the edges, so the warps stage H1, delta_2, delta_1 and X in shared memory and read transposed
// operands with ldmatrix.trans. Every CTA writes its own partial gradient; a second kernel folds
// the partials in a fixed order, so gradients are deterministic.
#include "sfg_internal.cuh"

namespace {

constexpr int kF = 16, kH = 64;
constexpr int OFF_W1 = 0, OFF_B1 = 1024, OFF_W2 = 1088, OFF_B2 = 5184, OFF_W3 = 5248,
              OFF_B3 = 5312, NP = 5313;
constexpr int kMlpBlock = 128;  // 4 warps

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint2 b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void* smem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}

struct Net {  // device pointers of one network
    const float* theta;
    const uint2* w1f;   // [8 n-tiles][32 lanes]
    const uint2* w2f;   // [8 n-tiles][4 k-steps][32 lanes]
    const uint2* w2tf;  // B fragments of W2^T, same shape
};

// Forward of 16 edges [e0, e0 + 16) of a warp. x: feature rows (FP32, 16 per row). Returns the
// post-ReLU layer outputs in accumulator layout (rows g and g + 8, columns 8j + 2t + {0, 1}) and
// y for rows g, g + 8 (valid in all four lanes of the row).
struct Tile {
    float h1[8][4], h2[8][4];
    uint32_t a1[4];
    float y0, y1;
};

__device__ __forceinline__ void forward_tile(const Net& net, const float* __restrict__ x,
                                             int64_t e0, int64_t ne, Tile& T) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t r0 = min(e0 + g, ne - 1), r1 = min(e0 + g + 8, ne - 1);
    const float2 x00 = *reinterpret_cast<const float2*>(x + r0 * kF + 2 * t);
    const float2 x10 = *reinterpret_cast<const float2*>(x + r1 * kF + 2 * t);
    const float2 x01 = *reinterpret_cast<const float2*>(x + r0 * kF + 8 + 2 * t);
    const float2 x11 = *reinterpret_cast<const float2*>(x + r1 * kF + 8 + 2 * t);
    T.a1[0] = pack_bf16(x00.x, x00.y);
    T.a1[1] = pack_bf16(x10.x, x10.y);
    T.a1[2] = pack_bf16(x01.x, x01.y);
    T.a1[3] = pack_bf16(x11.x, x11.y);
    const float* b1 = net.theta + OFF_B1;
    const float* b2 = net.theta + OFF_B2;
    const float* w3 = net.theta + OFF_W3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float c0 = b1[8 * j + 2 * t], c1 = b1[8 * j + 2 * t + 1];
        T.h1[j][0] = c0; T.h1[j][1] = c1; T.h1[j][2] = c0; T.h1[j][3] = c1;
        mma16816(T.h1[j], T.a1, net.w1f[j * 32 + lane]);
#pragma unroll
        for (int c = 0; c < 4; ++c) T.h1[j][c] = fmaxf(T.h1[j][c], 0.f);
    }
    uint32_t a2[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        a2[kk][0] = pack_bf16(T.h1[2 * kk][0], T.h1[2 * kk][1]);
        a2[kk][1] = pack_bf16(T.h1[2 * kk][2], T.h1[2 * kk][3]);
        a2[kk][2] = pack_bf16(T.h1[2 * kk + 1][0], T.h1[2 * kk + 1][1]);
        a2[kk][3] = pack_bf16(T.h1[2 * kk + 1][2], T.h1[2 * kk + 1][3]);
    }
    float y0 = 0.f, y1 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float c0 = b2[8 * j + 2 * t], c1 = b2[8 * j + 2 * t + 1];
        T.h2[j][0] = c0; T.h2[j][1] = c1; T.h2[j][2] = c0; T.h2[j][3] = c1;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) mma16816(T.h2[j], a2[kk], net.w2f[(j * 4 + kk) * 32 + lane]);
#pragma unroll
        for (int c = 0; c < 4; ++c) T.h2[j][c] = fmaxf(T.h2[j][c], 0.f);
        const float v0 = w3[8 * j + 2 * t], v1 = w3[8 * j + 2 * t + 1];
        y0 = fmaf(T.h2[j][0], v0, fmaf(T.h2[j][1], v1, y0));
        y1 = fmaf(T.h2[j][2], v0, fmaf(T.h2[j][3], v1, y1));
    }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
    T.y0 = y0 + net.theta[OFF_B3];
    T.y1 = y1 + net.theta[OFF_B3];
}

// ---- inference on the 5th-generation tensor cores (tcgen05, accumulators in TMEM) ----
// One CTA of 128 threads takes 128 edges at a time (the M of one MMA); each thread owns one row.
// Operands sit in shared memory in the K-major, non-swizzled core-matrix layout (8 rows x 16 bytes
// per core matrix; LBO = byte step along K, SBO = byte step between 8-row groups), as K = 16
// chunks. The A tile has five chunks: chunks 0-3 hold H1 (64 columns) and chunk 4 a constant
// (1, 1, 0, ..., 0) per row; chunk 0 also holds the BF16 features while layer 1 runs (H1 is
// written only after layer 1 has completed). The biases ride in the MMAs: the B rows facing the
// two constant columns hold b = hi + lo as two BF16 numbers (hi = BF16(b), lo = BF16(b - hi)), so
// the accumulator receives x W + b with b good to about 2^-16 relative.
//   layer 1: D = [x | 1 1 0..] [W1 ; b1_hi ; b1_lo ; 0..]           (2 MMAs, 128 x 64 x 16)
//   H1 = BF16(ReLU(D)) in one cvt.rn.relu.bf16x2 per column pair, written over chunks 0-3
//   layer 2: D = [H1 | 1 1 0..] [W2 ; b2_hi ; b2_lo ; 0..]          (5 MMAs)
//   y = sum_j ReLU(D_j) w3_j + b3 in FP32 by the owning thread.
// BF16 rounding points: features, W1, W2, H1 (as in the warp-level kernel). Completion of each MMA
// group is signalled through an mbarrier by tcgen05.commit; every wait on it is bounded.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);  // version 1, no swizzle
}

// kind::f16 instruction descriptor: D = F32 (bits 4-5), A = B = BF16 (bits 7-9, 10-12), both
// K-major, N / 8 at bit 17, M / 16 at bit 24.
constexpr uint32_t kIdescM128N64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) |
                                   ((128u >> 4) << 24);

__device__ __forceinline__ void umma_f16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(tmem), "l"(ad), "l"(bd), "r"(kIdescM128N64), "r"(acc) : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
    return done != 0;
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per thread)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_sync() {  // order tensor-core work and thread work across the CTA
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// bf16 index of element (row, k) of an R x KDIM K-major operand in the core-matrix layout
template <int KDIM>
__device__ __forceinline__ int core_idx(int row, int k) {
    return ((row >> 3) * (KDIM / 8) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

// BF16(ReLU(lo)) in the low half, BF16(ReLU(hi)) in the high half, round to nearest even
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

constexpr int kKA = 80;  // K of the A tile: H1 (64) + the constant chunk (16)
constexpr int kKB1 = 32; // K of layer 1's B: W1 (16) + bias chunk (16)

__global__ void __launch_bounds__(128, 6) k_mlp_forward_tc(const float* __restrict__ theta,
                                                         const float* __restrict__ x, int64_t ne,
                                                         float* __restrict__ out, int* __restrict__ err) {
    __shared__ __align__(1024) __nv_bfloat16 sA[128 * kKA];   // 20 KB
    __shared__ __align__(1024) __nv_bfloat16 sB1[kH * kKB1];  // W1 and b1 as N x K, 4 KB
    __shared__ __align__(1024) __nv_bfloat16 sB2[kH * kKA];   // W2 and b2 as N x K, 10 KB
    __shared__ __align__(16) float sw3[kH];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(64) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B operands: (n, k) = (output unit, input unit); the bias rows sit at k = K0 and K0 + 1
    auto split = [](float b, bool lo) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(b);
        return lo ? __float2bfloat16_rn(b - __bfloat162float(hi)) : hi;
    };
    for (int i = tid; i < kH * kKB1; i += 128) {
        const int h = i / kKB1, k = i % kKB1;
        sB1[core_idx<kKB1>(h, k)] = k < kF ? __float2bfloat16_rn(theta[OFF_W1 + k * kH + h])
                                  : k < kF + 2 ? split(theta[OFF_B1 + h], k == kF + 1)
                                               : __float2bfloat16_rn(0.f);
    }
    for (int i = tid; i < kH * kKA; i += 128) {
        const int j = i / kKA, k = i % kKA;
        sB2[core_idx<kKA>(j, k)] = k < kH ? __float2bfloat16_rn(theta[OFF_W2 + k * kH + j])
                                 : k < kH + 2 ? split(theta[OFF_B2 + j], k == kH + 1)
                                              : __float2bfloat16_rn(0.f);
    }
    if (tid < kH) sw3[tid] = theta[OFF_W3 + tid];
    {   // this row's constant chunk (1, 1, 0, ..., 0)
        const uint32_t one2 = pack_bf16(1.f, 1.f);
        *reinterpret_cast<uint4*>(&sA[core_idx<kKA>(tid, kH)]) = make_uint4(one2, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(&sA[core_idx<kKA>(tid, kH + 8)]) = make_uint4(0u, 0u, 0u, 0u);
    }
    const float b3 = theta[OFF_B3];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t a0 = smem_u32(sA), b10 = smem_u32(sB1), b20 = smem_u32(sB2);
    constexpr uint32_t kSboA = kKA / 8 * 128, kSboB1 = kKB1 / 8 * 128;
    uint32_t phase = 0;
    bool ok = true;
    const int64_t ntiles = (ne + 127) / 128;
    // this thread's feature row of the next tile, loaded one tile ahead so that the global
    // latency overlaps the current tile's MMAs
    float4 f[4];
    auto load_row = [&](int64_t tile) {
        const float4* xr = reinterpret_cast<const float4*>(x + min(tile * 128 + tid, ne - 1) * kF);
#pragma unroll
        for (int c = 0; c < 4; ++c) f[c] = xr[c];
    };
    if ((int64_t)blockIdx.x < ntiles) load_row(blockIdx.x);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t row = tile * 128 + tid;
        // features -> BF16 in chunk 0 (the previous tile's layer 2 has completed)
#pragma unroll
        for (int c = 0; c < 2; ++c)
            *reinterpret_cast<uint4*>(&sA[core_idx<kKA>(tid, 8 * c)]) =
                make_uint4(pack_bf16(f[2 * c].x, f[2 * c].y), pack_bf16(f[2 * c].z, f[2 * c].w),
                           pack_bf16(f[2 * c + 1].x, f[2 * c + 1].y), pack_bf16(f[2 * c + 1].z, f[2 * c + 1].w));
        if (tile + gridDim.x < ntiles) load_row(tile + gridDim.x);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_sync();  // also orders the previous tile's TMEM reads before this tile's MMAs
        if (tid == 0) {
            umma_f16(tmem, umma_desc(a0, 128, kSboA), umma_desc(b10, 128, kSboB1), 0);
            umma_f16(tmem, umma_desc(a0 + 256 * 4, 128, kSboA), umma_desc(b10 + 256, 128, kSboB1), 1);
            umma_commit(&mbar);
        }
        ok = __syncthreads_and(mbar_wait(&mbar, phase));  // one decision for the whole CTA
        phase ^= 1;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // H1 = BF16(ReLU(x W1 + b1)) over chunks 0-3, 32 columns at a time
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float v[32];
            tmem_ld32(taddr + 32 * half, v);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                *reinterpret_cast<uint4*>(&sA[core_idx<kKA>(tid, 32 * half + 8 * c)]) =
                    make_uint4(relu_bf16x2(v[8 * c], v[8 * c + 1]), relu_bf16x2(v[8 * c + 2], v[8 * c + 3]),
                               relu_bf16x2(v[8 * c + 4], v[8 * c + 5]), relu_bf16x2(v[8 * c + 6], v[8 * c + 7]));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_sync();
        if (tid == 0) {
#pragma unroll
            for (int c = 0; c < kKA / 16; ++c)
                umma_f16(tmem, umma_desc(a0 + 256 * c, 128, kSboA), umma_desc(b20 + 256 * c, 128, kSboA), c > 0);
            umma_commit(&mbar);
        }
        ok = __syncthreads_and(mbar_wait(&mbar, phase));
        phase ^= 1;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float y = 0.f;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float v[32];
            tmem_ld32(taddr + 32 * half, v);
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                const float4 w = *reinterpret_cast<const float4*>(&sw3[32 * half + j]);
                y = fmaf(fmaxf(v[j], 0.f), w.x, y);
                y = fmaf(fmaxf(v[j + 1], 0.f), w.y, y);
                y = fmaf(fmaxf(v[j + 2], 0.f), w.z, y);
                y = fmaf(fmaxf(v[j + 3], 0.f), w.w, y);
            }
        }
        if (row < ne) out[row] = y + b3;
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    tc_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(64) : "memory");
}


constexpr int kS64 = 72;  // shared-memory row stride (BF16) of the 64-wide tiles
constexpr int kS16 = 24;  // and of the 16-wide feature tile

// Gradient of L = (1/ne) sum (y - t)^2 over [0, ne): one partial per CTA, part[cta][NP + 1]
// (the last entry is the CTA's sum of squared errors).
__global__ void __launch_bounds__(kMlpBlock) k_mlp_fwdbwd(Net net, const float* __restrict__ x,
                                                          const float* __restrict__ target,
                                                          int64_t ne, float* __restrict__ part) {
    __shared__ __align__(16) __nv_bfloat16 sH1[64 * kS64];
    __shared__ __align__(16) __nv_bfloat16 sD2[64 * kS64];
    __shared__ __align__(16) __nv_bfloat16 sD1[64 * kS64];
    __shared__ __align__(16) __nv_bfloat16 sX[64 * kS16];
    __shared__ float sred[4][3 * kH + 2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const float* w3 = net.theta + OFF_W3;
    const float inv_n = 1.0f / (float)ne;
    float acc2[8][4], acc1[2][4];
    float db1[16], db2[16], dw3[16];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc2[j][c] = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc1[0][c] = acc1[1][c] = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) db1[i] = db2[i] = dw3[i] = 0.f;
    float db3 = 0.f, sse = 0.f;

    for (int64_t c0 = (int64_t)blockIdx.x * 64; c0 < ne; c0 += (int64_t)gridDim.x * 64) {
        const int64_t e0 = c0 + warp * 16;
        Tile T;
        forward_tile(net, x, e0, ne, T);
        const bool v0 = e0 + g < ne, v1 = e0 + g + 8 < ne;
        const float r0 = v0 ? T.y0 - target[e0 + g] : 0.f;
        const float r1 = v1 ? T.y1 - target[e0 + g + 8] : 0.f;
        if (t == 0) {
            sse = fmaf(r0, r0, fmaf(r1, r1, sse));
            db3 += 2.f * (r0 + r1) * inv_n;
        }
        const float d30 = 2.f * r0 * inv_n, d31 = 2.f * r1 * inv_n;
        // delta_2 = delta_3 w3 (.) [z2 > 0]; db2, dw3
        float d2[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float v0w = w3[8 * j + 2 * t], v1w = w3[8 * j + 2 * t + 1];
            dw3[2 * j] += T.h2[j][0] * d30 + T.h2[j][2] * d31;
            dw3[2 * j + 1] += T.h2[j][1] * d30 + T.h2[j][3] * d31;
            d2[j][0] = T.h2[j][0] > 0.f ? d30 * v0w : 0.f;
            d2[j][1] = T.h2[j][1] > 0.f ? d30 * v1w : 0.f;
            d2[j][2] = T.h2[j][2] > 0.f ? d31 * v0w : 0.f;
            d2[j][3] = T.h2[j][3] > 0.f ? d31 * v1w : 0.f;
            db2[2 * j] += d2[j][0] + d2[j][2];
            db2[2 * j + 1] += d2[j][1] + d2[j][3];
        }
        uint32_t ad2[4][4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            ad2[kk][0] = pack_bf16(d2[2 * kk][0], d2[2 * kk][1]);
            ad2[kk][1] = pack_bf16(d2[2 * kk][2], d2[2 * kk][3]);
            ad2[kk][2] = pack_bf16(d2[2 * kk + 1][0], d2[2 * kk + 1][1]);
            ad2[kk][3] = pack_bf16(d2[2 * kk + 1][2], d2[2 * kk + 1][3]);
        }
        // delta_1 = (delta_2 W2^T) (.) [z1 > 0]; db1
        float d1[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
#pragma unroll
            for (int c = 0; c < 4; ++c) d1[j][c] = 0.f;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) mma16816(d1[j], ad2[kk], net.w2tf[(j * 4 + kk) * 32 + lane]);
#pragma unroll
            for (int c = 0; c < 4; ++c) d1[j][c] = T.h1[j][c] > 0.f ? d1[j][c] : 0.f;
            db1[2 * j] += d1[j][0] + d1[j][2];
            db1[2 * j + 1] += d1[j][1] + d1[j][3];
        }
        // stage H1, delta_2, delta_1 and X (BF16) for the contractions over edges
        const int er0 = warp * 16 + g, er1 = er0 + 8;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = 8 * j + 2 * t;
            *reinterpret_cast<uint32_t*>(&sH1[er0 * kS64 + col]) = v0 ? pack_bf16(T.h1[j][0], T.h1[j][1]) : 0u;
            *reinterpret_cast<uint32_t*>(&sH1[er1 * kS64 + col]) = v1 ? pack_bf16(T.h1[j][2], T.h1[j][3]) : 0u;
            *reinterpret_cast<uint32_t*>(&sD2[er0 * kS64 + col]) = pack_bf16(d2[j][0], d2[j][1]);
            *reinterpret_cast<uint32_t*>(&sD2[er1 * kS64 + col]) = pack_bf16(d2[j][2], d2[j][3]);
            *reinterpret_cast<uint32_t*>(&sD1[er0 * kS64 + col]) = pack_bf16(d1[j][0], d1[j][1]);
            *reinterpret_cast<uint32_t*>(&sD1[er1 * kS64 + col]) = pack_bf16(d1[j][2], d1[j][3]);
        }
        *reinterpret_cast<uint32_t*>(&sX[er0 * kS16 + 2 * t]) = v0 ? T.a1[0] : 0u;
        *reinterpret_cast<uint32_t*>(&sX[er1 * kS16 + 2 * t]) = v1 ? T.a1[1] : 0u;
        *reinterpret_cast<uint32_t*>(&sX[er0 * kS16 + 8 + 2 * t]) = v0 ? T.a1[2] : 0u;
        *reinterpret_cast<uint32_t*>(&sX[er1 * kS16 + 8 + 2 * t]) = v1 ? T.a1[3] : 0u;
        __syncthreads();
        // dW2[j][i] = sum_e H1[e][j] delta_2[e][i]: this warp owns rows j in [16 warp, 16 warp + 16)
        // dW1[f][j] = sum_e X[e][f] delta_1[e][j]: this warp owns columns j in [16 warp, 16 warp + 16)
        const int mat = lane >> 3, rr = lane & 7;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            const int eb = ks * 16;
            uint32_t a[4];
            ldsm_x4_trans(a, &sH1[(eb + rr + 8 * (mat >> 1)) * kS64 + warp * 16 + 8 * (mat & 1)]);
#pragma unroll
            for (int nt = 0; nt < 8; nt += 2) {
                uint32_t b[4];
                ldsm_x4_trans(b, &sD2[(eb + rr + 8 * (mat & 1)) * kS64 + nt * 8 + 8 * (mat >> 1)]);
                mma16816(acc2[nt], a, make_uint2(b[0], b[1]));
                mma16816(acc2[nt + 1], a, make_uint2(b[2], b[3]));
            }
            uint32_t ax[4], bx[4];
            ldsm_x4_trans(ax, &sX[(eb + rr + 8 * (mat >> 1)) * kS16 + 8 * (mat & 1)]);
            ldsm_x4_trans(bx, &sD1[(eb + rr + 8 * (mat & 1)) * kS64 + warp * 16 + 8 * (mat >> 1)]);
            mma16816(acc1[0], ax, make_uint2(bx[0], bx[1]));
            mma16816(acc1[1], ax, make_uint2(bx[2], bx[3]));
        }
        __syncthreads();
    }

    // write this CTA's partial gradient
    float* P = part + (size_t)blockIdx.x * (NP + 1);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int j = warp * 16 + g, i = nt * 8 + 2 * t;
        P[OFF_W2 + j * kH + i] = acc2[nt][0];
        P[OFF_W2 + j * kH + i + 1] = acc2[nt][1];
        P[OFF_W2 + (j + 8) * kH + i] = acc2[nt][2];
        P[OFF_W2 + (j + 8) * kH + i + 1] = acc2[nt][3];
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int j = warp * 16 + q * 8 + 2 * t;
        P[OFF_W1 + g * kH + j] = acc1[q][0];
        P[OFF_W1 + g * kH + j + 1] = acc1[q][1];
        P[OFF_W1 + (g + 8) * kH + j] = acc1[q][2];
        P[OFF_W1 + (g + 8) * kH + j + 1] = acc1[q][3];
    }
    // column sums over the rows held by lanes with the same t, then over warps
#pragma unroll
    for (int i = 0; i < 16; ++i)
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            db1[i] += __shfl_xor_sync(0xffffffffu, db1[i], o);
            db2[i] += __shfl_xor_sync(0xffffffffu, db2[i], o);
            dw3[i] += __shfl_xor_sync(0xffffffffu, dw3[i], o);
        }
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
        db3 += __shfl_xor_sync(0xffffffffu, db3, o);
        sse += __shfl_xor_sync(0xffffffffu, sse, o);
    }
    if (lane < 4) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            sred[warp][8 * j + 2 * t] = db1[2 * j];
            sred[warp][8 * j + 2 * t + 1] = db1[2 * j + 1];
            sred[warp][kH + 8 * j + 2 * t] = db2[2 * j];
            sred[warp][kH + 8 * j + 2 * t + 1] = db2[2 * j + 1];
            sred[warp][2 * kH + 8 * j + 2 * t] = dw3[2 * j];
            sred[warp][2 * kH + 8 * j + 2 * t + 1] = dw3[2 * j + 1];
        }
        if (lane == 0) {
            sred[warp][3 * kH] = db3;
            sred[warp][3 * kH + 1] = sse;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * kH + 2; i += kMlpBlock) {
        const float s = sred[0][i] + sred[1][i] + sred[2][i] + sred[3][i];
        if (i < kH) P[OFF_B1 + i] = s;
        else if (i < 2 * kH) P[OFF_B2 + i - kH] = s;
        else if (i < 3 * kH) P[OFF_W3 + i - 2 * kH] = s;
        else if (i == 3 * kH) P[OFF_B3] = s;
        else P[NP] = s;
    }
}

// grad[i] = sum over CTAs (in order) of part[cta][i]; loss = sum of squared errors / ne
__global__ void k_mlp_fold(const float* __restrict__ part, int nparts, int64_t ne,
                           float* __restrict__ grad, double* __restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > NP) return;
    double s = 0.0;
    for (int c = 0; c < nparts; ++c) s += (double)part[(size_t)c * (NP + 1) + i];
    if (i < NP) grad[i] = (float)s;
    else if (loss) *loss = s / (double)ne;
}

__global__ void k_mlp_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ grad, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// B-operand fragments of W1, W2 and W2^T from the FP32 parameters.
__global__ void k_mlp_frags(const float* __restrict__ theta, uint2* __restrict__ w1f,
                            uint2* __restrict__ w2f, uint2* __restrict__ w2tf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // [0, 256) W1, then 1024 each W2, W2^T
    const float* W1 = theta + OFF_W1;
    const float* W2 = theta + OFF_W2;
    if (i < 256) {
        const int j = i >> 5, lane = i & 31, g = lane >> 2, t = lane & 3, n = 8 * j + g;
        w1f[i] = make_uint2(pack_bf16(W1[(2 * t) * kH + n], W1[(2 * t + 1) * kH + n]),
                            pack_bf16(W1[(2 * t + 8) * kH + n], W1[(2 * t + 9) * kH + n]));
    } else if (i < 256 + 1024) {
        const int q = i - 256, lane = q & 31, kk = (q >> 5) & 3, j = q >> 7, g = lane >> 2, t = lane & 3;
        const int n = 8 * j + g, k0 = 16 * kk + 2 * t;
        w2f[q] = make_uint2(pack_bf16(W2[k0 * kH + n], W2[(k0 + 1) * kH + n]),
                            pack_bf16(W2[(k0 + 8) * kH + n], W2[(k0 + 9) * kH + n]));
    } else if (i < 256 + 2048) {
        const int q = i - 1280, lane = q & 31, kk = (q >> 5) & 3, j = q >> 7, g = lane >> 2, t = lane & 3;
        const int n = 8 * j + g, k0 = 16 * kk + 2 * t;  // B[k][n] = W2[n][k]
        w2tf[q] = make_uint2(pack_bf16(W2[n * kH + k0], W2[n * kH + k0 + 1]),
                             pack_bf16(W2[n * kH + k0 + 8], W2[n * kH + k0 + 9]));
    }
}

// Kaiming-uniform initial weights from the counter-based generator, biases 0.
__global__ void k_mlp_init(uint64_t seed, float* __restrict__ theta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    float b = 0.f;
    if (i < OFF_B1) b = sqrtf(6.f / kF);
    else if (i >= OFF_W2 && i < OFF_B2) b = sqrtf(6.f / kH);
    else if (i >= OFF_W3 && i < OFF_B3) b = sqrtf(6.f / kH);
    const uint64_t s0 = sfg_splitmix64(seed);
    const uint64_t o = sfg_splitmix64(s0 + (uint64_t)i * 0x9E3779B97F4A7C15ull);
    const double u = (double)(o >> 11) * 0x1.0p-53;
    theta[i] = b > 0.f ? (float)((2.0 * u - 1.0) * (double)b) : 0.f;
}

// Feature rows (see include/sfg.h) of the listed edges from their projected-embedding distances.
__global__ void k_mlp_features(int64_t ne, const int32_t* __restrict__ ids,
                               const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                               const float* __restrict__ ew, const double* __restrict__ deg,
                               const int32_t* __restrict__ row_ptr, const float* __restrict__ sg,
                               const float* __restrict__ sp, float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = ids[i], p = eu[e], q = ev[e];
        const float lp = logf((float)deg[p]), lq = logf((float)deg[q]);
        const float g = sg[i], s = sp[i];
        float f[kF];
        f[0] = logf(ew[e]);
        f[1] = lp + lq;
        f[2] = fabsf(lp - lq);
        f[3] = logf(g + 1e-30f);
        f[4] = logf(s + 1e-30f);
        f[5] = logf(s + 1e-30f) - logf(g + 1e-30f);
        f[6] = logf((float)(row_ptr[p + 1] - row_ptr[p]) * (float)(row_ptr[q + 1] - row_ptr[q]));
        f[7] = logf(g + s + 1e-30f);
#pragma unroll
        for (int k = 8; k < kF; ++k) f[k] = 0.f;
        float4* o4 = reinterpret_cast<float4*>(out + i * kF);
#pragma unroll
        for (int k = 0; k < kF / 4; ++k) o4[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
    }
}

}  // namespace

struct sfg_mlp {
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    uint2 *w1f = nullptr, *w2f = nullptr, *w2tf = nullptr;
    int64_t step = 0;
    cudaStream_t stream = nullptr;
    int device = -1;
};

static Net net_of(const sfg_mlp* n) { return Net{n->theta, n->w1f, n->w2f, n->w2tf}; }

static sfg_status refresh_frags(sfg_ctx* ctx, sfg_mlp* n) {
    k_mlp_frags<<<ceil_div_u(256 + 2048, 256), 256, 0, ctx->stream>>>(n->theta, n->w1f, n->w2f, n->w2tf);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_mlp_frags");
    return SFG_OK;
}

static void mlp_free(sfg_mlp* n) {
    if (!n) return;
    SfgDeviceGuard guard(n->device);
    void* ptrs[] = {n->theta, n->m, n->v, n->grad, n->w1f, n->w2f, n->w2tf};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, n->stream);
    delete n;
}

// gradient (and loss) of the network on [feats, targets) into n->grad
static sfg_status mlp_grad(sfg_ctx* ctx, sfg_mlp* n, const float* feats, const float* targets,
                           int64_t ne, double* loss_dev) {
    const int grid = (int)std::min<int64_t>((ne + 63) / 64,
                                            (int64_t)sfg_grid(ctx, (const void*)k_mlp_fwdbwd,
                                                              kMlpBlock, 0, ne * 2));
    Scratch s(ctx);
    float* part;
    SFG_TRY(s.get(&part, (size_t)grid * (NP + 1)));
    sfg_tic(ctx, "mlp_fwdbwd");
    k_mlp_fwdbwd<<<grid, kMlpBlock, 0, ctx->stream>>>(net_of(n), feats, targets, ne, part);
    sfg_toc(ctx);
    k_mlp_fold<<<ceil_div_u(NP + 1, 256), 256, 0, ctx->stream>>>(part, grid, ne, n->grad, loss_dev);
    ctx->launches += 2;
    SFG_LAUNCH_CHECK(ctx, "k_mlp_fwdbwd");
    return SFG_OK;
}

sfg_status sfg_mlp_forward_impl(sfg_ctx* ctx, const sfg_mlp* net, const float* feats, int64_t ne,
                                float* out) {
    if (ne == 0) return SFG_OK;
    Scratch s(ctx);
    int* err;
    SFG_TRY(s.get(&err, 1));
    SFG_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
    const int64_t ntiles = (ne + 127) / 128;
    // One wave of resident CTAs, counted from the kernel's registers and static shared memory
    // (each CTA also holds 64 of the SM's 512 TMEM columns, so at most 8 fit); kept per context,
    // i.e. per device.
    const auto key = std::make_tuple((const void*)k_mlp_forward_tc, 128, (size_t)0);
    int per_sm = 0;
    if (auto it = ctx->occupancy.find(key); it != ctx->occupancy.end()) {
        per_sm = it->second;
    } else {
        SFG_CUDA(ctx, cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                           (int)cudaSharedmemCarveoutMaxShared));
        cudaFuncAttributes fa;
        SFG_CUDA(ctx, cudaFuncGetAttributes(&fa, k_mlp_forward_tc));
        int regs_sm = 0, smem_sm = 0, smem_rsv = 0;
        SFG_CUDA(ctx, cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, ctx->device));
        SFG_CUDA(ctx, cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
        SFG_CUDA(ctx, cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, ctx->device));
        const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;  // allocated per warp in units of 256
        const int by_regs = regs_sm / (warp_regs * 4);
        const int by_smem = smem_sm / ((int)fa.sharedSizeBytes + smem_rsv);
        per_sm = std::max(1, std::min({by_regs, by_smem, 512 / 64}));
        ctx->occupancy.emplace(key, per_sm);
    }
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)ctx->num_sms * per_sm);
    sfg_tic(ctx, "mlp_forward");
    k_mlp_forward_tc<<<grid, 128, 0, ctx->stream>>>(net->theta, feats, ne, out, err);
    sfg_toc(ctx);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_mlp_forward_tc");
    int h = 0;
    SFG_CUDA(ctx, cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (h) return sfg_fail(ctx, SFG_ETIMEOUT, "MLP forward: a tensor-core completion wait ran out");
    return SFG_OK;
}

sfg_status sfg_edge_features_impl(sfg_ctx* ctx, const sfg_graph* LG, const sfg_graph* LP, int K,
                                  int steps, double omega, uint64_t seed, sfg_dtype storage,
                                  const int32_t* ids, int64_t ne, float* feats) {
    if (ne == 0) return SFG_OK;
    Scratch s(ctx);
    float *sg, *sp;
    SFG_TRY(s.get(&sg, ne));
    SFG_TRY(s.get(&sp, ne));
    SFG_TRY(sfg_filter_score_impl(ctx, LG, LP, K, steps, omega, seed, storage, ids, ne, SFG_SCORE_G, sg));
    SFG_TRY(sfg_filter_score_impl(ctx, LG, LP, K, steps, omega, seed, storage, ids, ne, SFG_SCORE_P, sp));
    k_mlp_features<<<sfg_grid(ctx, (const void*)k_mlp_features, 256, 0, ne), 256, 0, ctx->stream>>>(
        ne, ids, LG->eu, LG->ev, LG->ew, LG->deg, LG->row_ptr, sg, sp, feats);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_mlp_features");
    return SFG_OK;
}

extern "C" {

sfg_status sfg_mlp_create(sfg_ctx* ctx, uint64_t seed, sfg_mlp** out) {
    if (!ctx || !out) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    *out = nullptr;
    sfg_mlp* n = new sfg_mlp();
    n->stream = ctx->stream;
    n->device = ctx->device;
    sfg_status st = SFG_OK;
    auto A = [&](void** p, size_t bytes) {
        if (st == SFG_OK) st = sfg_alloc(ctx, p, bytes);
    };
    A((void**)&n->theta, 4 * NP);
    A((void**)&n->m, 4 * NP);
    A((void**)&n->v, 4 * NP);
    A((void**)&n->grad, 4 * NP);
    A((void**)&n->w1f, sizeof(uint2) * 256);
    A((void**)&n->w2f, sizeof(uint2) * 1024);
    A((void**)&n->w2tf, sizeof(uint2) * 1024);
    if (st != SFG_OK) {
        mlp_free(n);
        return st;
    }
    SFG_CUDA(ctx, cudaMemsetAsync(n->m, 0, 4 * NP, ctx->stream));
    SFG_CUDA(ctx, cudaMemsetAsync(n->v, 0, 4 * NP, ctx->stream));
    k_mlp_init<<<ceil_div_u(NP, 256), 256, 0, ctx->stream>>>(seed, n->theta);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_mlp_init");
    SFG_TRY(refresh_frags(ctx, n));
    *out = n;
    return SFG_OK;
}

void sfg_mlp_destroy(sfg_mlp* net) { mlp_free(net); }

sfg_status sfg_mlp_params(sfg_ctx* ctx, const sfg_mlp* net, float* theta_out) {
    if (!ctx || !net) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    SFG_TRY(sfg_check_dev(ctx, theta_out, "theta_out"));
    SFG_CUDA(ctx, cudaMemcpyAsync(theta_out, net->theta, 4 * NP, cudaMemcpyDeviceToDevice, ctx->stream));
    return SFG_OK;
}

sfg_status sfg_mlp_set_params(sfg_ctx* ctx, sfg_mlp* net, const float* theta) {
    if (!ctx || !net) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    SFG_TRY(sfg_check_dev(ctx, theta, "theta"));
    SFG_CUDA(ctx, cudaMemcpyAsync(net->theta, theta, 4 * NP, cudaMemcpyDeviceToDevice, ctx->stream));
    SFG_CUDA(ctx, cudaMemsetAsync(net->m, 0, 4 * NP, ctx->stream));
    SFG_CUDA(ctx, cudaMemsetAsync(net->v, 0, 4 * NP, ctx->stream));
    net->step = 0;
    return refresh_frags(ctx, net);
}

sfg_status sfg_mlp_forward(sfg_ctx* ctx, const sfg_mlp* net, const float* feats, int64_t ne,
                           float* out) {
    if (!ctx || !net) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (ne < 0) return sfg_fail(ctx, SFG_EINVAL, "ne must be >= 0");
    if (ne == 0) return SFG_OK;
    SFG_TRY(sfg_check_dev(ctx, feats, "feats"));
    SFG_TRY(sfg_check_dev(ctx, out, "out"));
    return sfg_mlp_forward_impl(ctx, net, feats, ne, out);
}

sfg_status sfg_mlp_gradient(sfg_ctx* ctx, sfg_mlp* net, const float* feats, const float* targets,
                            int64_t ne, float* grad_out, double* loss_host) {
    if (!ctx || !net) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (ne < 1) return sfg_fail(ctx, SFG_EINVAL, "ne must be >= 1");
    SFG_TRY(sfg_check_dev(ctx, feats, "feats"));
    SFG_TRY(sfg_check_dev(ctx, targets, "targets"));
    Scratch s(ctx);
    double* loss;
    SFG_TRY(s.get(&loss, 1));
    SFG_TRY(mlp_grad(ctx, net, feats, targets, ne, loss));
    if (grad_out) {
        SFG_TRY(sfg_check_dev(ctx, grad_out, "grad_out"));
        SFG_CUDA(ctx, cudaMemcpyAsync(grad_out, net->grad, 4 * NP, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (loss_host) {
        SFG_CUDA(ctx, cudaMemcpyAsync(loss_host, loss, 8, cudaMemcpyDeviceToHost, ctx->stream));
        SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return SFG_OK;
}

sfg_status sfg_mlp_train(sfg_ctx* ctx, sfg_mlp* net, const float* feats, const float* targets,
                         int64_t ne, int64_t batch, int epochs, double lr, double* loss_host) {
    if (!ctx || !net) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (ne < 1 || batch < 1 || epochs < 0 || !(lr > 0.0))
        return sfg_fail(ctx, SFG_EINVAL, "bad training arguments");
    SFG_TRY(sfg_check_dev(ctx, feats, "feats"));
    SFG_TRY(sfg_check_dev(ctx, targets, "targets"));
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; ep < epochs; ++ep)
        for (int64_t i = 0; i < ne; i += batch) {
            const int64_t nb = std::min(batch, ne - i);
            SFG_TRY(mlp_grad(ctx, net, feats + i * kF, targets + i, nb, nullptr));
            net->step += 1;
            const float c1 = 1.f - powf(b1, (float)net->step), c2 = 1.f - powf(b2, (float)net->step);
            k_mlp_adam<<<ceil_div_u(NP, 256), 256, 0, ctx->stream>>>(net->theta, net->m, net->v,
                                                                     net->grad, (float)lr, b1, b2,
                                                                     1e-8f, c1, c2);
            ++ctx->launches;
            SFG_LAUNCH_CHECK(ctx, "k_mlp_adam");
            SFG_TRY(refresh_frags(ctx, net));
        }
    if (loss_host) {
        Scratch s(ctx);
        double* loss;
        SFG_TRY(s.get(&loss, 1));
        SFG_TRY(mlp_grad(ctx, net, feats, targets, ne, loss));
        SFG_CUDA(ctx, cudaMemcpyAsync(loss_host, loss, 8, cudaMemcpyDeviceToHost, ctx->stream));
        SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return SFG_OK;
}

sfg_status sfg_edge_features(sfg_ctx* ctx, const sfg_graph* LG, const sfg_graph* LP, int K,
                             int steps, double omega, uint64_t seed, sfg_dtype storage,
                             const int32_t* edge_ids, int64_t ne, float* feats_out) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!LG || !LP || LG->n != LP->n) return sfg_fail(ctx, SFG_EINVAL, "bad graphs");
    if (!sfg_k_supported(K, storage))
        return sfg_fail(ctx, SFG_EUNSUPPORTED, "K=%d unsupported for dtype %d", K, (int)storage);
    if (steps < 0 || !(omega > 0.0 && omega <= 1.0) || ne < 0)
        return sfg_fail(ctx, SFG_EINVAL, "bad arguments");
    if (ne == 0) return SFG_OK;
    SFG_TRY(sfg_check_dev(ctx, edge_ids, "edge_ids"));
    SFG_TRY(sfg_check_dev(ctx, feats_out, "feats_out"));
    return sfg_edge_features_impl(ctx, LG, LP, K, steps, omega, seed, storage, edge_ids, ne, feats_out);
}

}  // extern "C"
