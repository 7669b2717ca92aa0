// Learned edge-proposal scorer (an addition to the paper's method; the proposals it makes are
// rescored by the plain method before selection): per-edge features from a short embedding and a
// 16 -> 64 -> 64 -> 1 ReLU network, evaluated (k_mlp_forward_tc) and trained (k_mlp_fwdbwd_tc,
// forward and backward) on the 5th-generation tensor cores: BF16 operands in shared memory, FP32
// accumulators in TMEM, completion through mbarriers with bounded waits. Adam in FP32 on the
// CUDA cores. Every CTA of the training kernel writes its own partial gradient and a second
// kernel folds the partials in a fixed order, so gradients are deterministic.
#include "sfg_internal.cuh"

namespace {

constexpr int kF = 16, kH = 64;
constexpr int OFF_W1 = 0, OFF_B1 = 1024, OFF_W2 = 1088, OFF_B2 = 5184, OFF_W3 = 5248,
              OFF_B3 = 5312, NP = 5313;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
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
// BF16 rounding points: features, W1, W2, H1. Completion of each MMA
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

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the mbarrier phase, giving up after about two seconds
__device__ __forceinline__ bool mbar_wait_timed(uint64_t* mbar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    uint32_t done = 0;
    while (true) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
        if (done) return true;
        if (global_ns() - t0 > 2000000000ull) return false;
    }
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
                                                         float* __restrict__ out, int* __restrict__ err,
                                                         int withhold) {
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
        if (tid == 0 && !withhold) {
            umma_f16(tmem, umma_desc(a0, 128, kSboA), umma_desc(b10, 128, kSboB1), 0);
            umma_f16(tmem, umma_desc(a0 + 256 * 4, 128, kSboA), umma_desc(b10 + 256, 128, kSboB1), 1);
            umma_commit(&mbar);
        }
        ok = __syncthreads_and(mbar_wait_timed(&mbar, phase));  // one decision for the whole CTA
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
        if (tid == 0 && !withhold) {
#pragma unroll
            for (int c = 0; c < kKA / 16; ++c)
                umma_f16(tmem, umma_desc(a0 + 256 * c, 128, kSboA), umma_desc(b20 + 256 * c, 128, kSboA), c > 0);
            umma_commit(&mbar);
        }
        ok = __syncthreads_and(mbar_wait_timed(&mbar, phase));
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
    if (!ok && tid == 0) {
        atomicExch(err, 1);
        mbar_wait_timed(&mbar, phase ^ 1);  // the group in flight completes before TMEM is released
    }
    tc_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(64) : "memory");
}


// ---- training on the 5th-generation tensor cores ----
// Gradient of L = (1/ne) sum (y - t)^2, one CTA of 128 threads per 128-edge tile (thread r owns
// edge row r = TMEM lane r), the tiles of a CTA in grid-stride order. Shared-memory operands, all
// BF16 in the K-major, non-swizzled core-matrix layout (8 rows x 16 bytes per core matrix):
//   sA  (128 x 96): H1 (columns 0-63) | X, the features (64-79) | constant chunk (1, 1, 0, ..) (80-95)
//   sD  (128 x 128): delta_2 (columns 0-63) | delta_1 (64-127)
//   sB1 (64 x 32): layer-1 B, (n = unit, k) = [W1 | b1_hi, b1_lo, 0 ..]
//   sB2 (64 x 96): layer-2 B, (n = unit j, k) = [W2 (k = i) | 0 (facing X) | b2_hi, b2_lo, 0 ..]
//   sB2T (64 x 64): (n = i, k = j) = W2[i][j], the B operand of delta_1 = delta_2 W2^T
// Per tile, each step an MMA group signalled through one mbarrier (waits bounded by a clock):
//   z1 = [X | 1] [W1; b1]               (A = sA columns 64-95, K = 32)   -> TMEM columns 0-63
//   H1 = BF16(ReLU(z1)) into sA; z2 = [H1 | X | 1] [W2; 0; b2]  (K = 96) -> TMEM columns 0-63
//   y = ReLU(z2) w3 + b3 (FP32, per thread); delta_3 = 2 (y - t) / ne; delta_2 = delta_3 w3 (.) [z2 > 0]
//   delta_1 = (delta_2 W2^T) (.) [z1 > 0]        (A = sD columns 0-63)   -> TMEM columns 0-63
//   G += [delta_2 | delta_1]^T [H1 | X | 1]      (K = the tile's 128 rows) -> TMEM columns 64-159
// The last product reads sD and sA as MN-major operands (the rows of the tile are its K), so the
// weight gradients need no transposed copies: G rows 0-63 (j) x columns 0-63 (i) = dW2[i][j],
// column 80 = db2[j]; G rows 64-127 (i) x columns 64-79 (f) = dW1[f][i], column 80 = db1[i]. G
// accumulates over the CTA's tiles in TMEM; dw3 = sum h2 delta_3 and db3 = sum delta_3 accumulate
// per thread in FP32. Each CTA writes its partial gradient; k_mlp_fold adds them in CTA order.
// BF16 rounding points: features, W1, W2, H1, delta_2, delta_1 (as in the inference kernel).
// kind::f16 instruction descriptor: D = F32, A = B = BF16, operand majors (0: K-major, 1: MN-major)
// at bits 15 (A) and 16 (B), N / 8 at bit 17, M / 16 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16_id(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                            uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
}

// Descriptor of an MN-major operand (no swizzle): the byte step between 8-row groups along K goes
// in the leading-byte-offset field and the step between 8-element groups along M (or N) in the
// stride-byte-offset field -- the roles the two fields have for a K-major operand swapped.
__device__ __forceinline__ uint64_t umma_desc_mn(uint32_t addr, uint32_t mn, uint32_t kg) {
    return umma_desc(addr, kg, mn);
}

constexpr int kTA = 96, kTD = 128, kTB1 = 32;
constexpr int kTColsTmem = 256;  // layer accumulator (64) + gradient (96), rounded to a power of two
constexpr size_t kTrainSmA = 128 * kTA * 2, kTrainSmD = 128 * kTD * 2, kTrainSmB1 = kH * kTB1 * 2,
                 kTrainSmB2 = kH * kTA * 2, kTrainSmB2T = kH * kH * 2;
constexpr size_t kTrainSmem = kTrainSmA + kTrainSmD + kTrainSmB1 + kTrainSmB2 + kTrainSmB2T + 1024;  // + alignment

__global__ void __launch_bounds__(128, 2)
    k_mlp_fwdbwd_tc(const float* __restrict__ theta, const float* __restrict__ x,
                    const float* __restrict__ target, int64_t ne, float* __restrict__ part,
                    int* __restrict__ err, int withhold) {
    extern __shared__ __align__(1024) uint8_t dsm[];
    uint8_t* base = dsm + ((1024 - (smem_u32(dsm) & 1023)) & 1023);  // 1024-byte aligned
    __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(base);
    __nv_bfloat16* sD = reinterpret_cast<__nv_bfloat16*>(base + kTrainSmA);
    __nv_bfloat16* sB1 = reinterpret_cast<__nv_bfloat16*>(base + kTrainSmA + kTrainSmD);
    __nv_bfloat16* sB2 = reinterpret_cast<__nv_bfloat16*>(base + kTrainSmA + kTrainSmD + kTrainSmB1);
    __nv_bfloat16* sB2T = reinterpret_cast<__nv_bfloat16*>(base + kTrainSmA + kTrainSmD + kTrainSmB1 + kTrainSmB2);
    __shared__ __align__(16) float sw3[kH];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(kTColsTmem) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&mbar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    auto split = [](float b, bool lo) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(b);
        return lo ? __float2bfloat16_rn(b - __bfloat162float(hi)) : hi;
    };
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    for (int i = tid; i < kH * kTB1; i += 128) {
        const int h = i / kTB1, k = i % kTB1;
        sB1[core_idx<kTB1>(h, k)] = k < kF ? __float2bfloat16_rn(theta[OFF_W1 + k * kH + h])
                                  : k < kF + 2 ? split(theta[OFF_B1 + h], k == kF + 1) : zero;
    }
    for (int i = tid; i < kH * kTA; i += 128) {
        const int j = i / kTA, k = i % kTA;
        sB2[core_idx<kTA>(j, k)] = k < kH ? __float2bfloat16_rn(theta[OFF_W2 + k * kH + j])
                                 : (k == 80 || k == 81) ? split(theta[OFF_B2 + j], k == 81) : zero;
    }
    for (int i = tid; i < kH * kH; i += 128) {
        const int a = i / kH, b = i % kH;   // (n = i, k = j) = W2[i][j]
        sB2T[core_idx<kH>(a, b)] = __float2bfloat16_rn(theta[OFF_W2 + a * kH + b]);
    }
    if (tid < kH) sw3[tid] = theta[OFF_W3 + tid];
    {   // this row's constant chunk (1, 1, 0, ..., 0) at columns 80-95
        const uint32_t one2 = pack_bf16(1.f, 1.f);
        *reinterpret_cast<uint4*>(&sA[core_idx<kTA>(tid, 80)]) = make_uint4(one2, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(&sA[core_idx<kTA>(tid, 88)]) = make_uint4(0u, 0u, 0u, 0u);
    }
    const float b3 = theta[OFF_B3];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    const uint32_t acc_z = tmem + lane_off, acc_g = tmem + lane_off + 64;
    const uint32_t a0 = smem_u32(sA), d0 = smem_u32(sD), b10 = smem_u32(sB1), b20 = smem_u32(sB2),
                   bt0 = smem_u32(sB2T);
    constexpr uint32_t kSboA = kTA / 8 * 128, kSboD = kTD / 8 * 128, kSboB1 = kTB1 / 8 * 128,
                       kSboB2T = kH / 8 * 128;
    constexpr uint32_t kId1 = idesc_f16(128, 64, 0, 0), kIdG = idesc_f16(128, 96, 1, 1);
    uint32_t phase = 0;
    bool ok = true;
    const float inv_n = 1.0f / (float)ne;
    float gw3[kH];
#pragma unroll
    for (int j = 0; j < kH; ++j) gw3[j] = 0.f;
    float gb3 = 0.f, sse = 0.f;
    const int64_t ntiles = (ne + 127) / 128;
    float4 f[4];
    auto load_row = [&](int64_t tile) {
        const float4* xr = reinterpret_cast<const float4*>(x + min(tile * 128 + tid, ne - 1) * kF);
#pragma unroll
        for (int c = 0; c < 4; ++c) f[c] = xr[c];
    };
    auto step = [&](auto&& issue) {  // one MMA group: issue, commit, bounded wait (CTA-wide)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_sync();
        if (tid == 0 && !withhold) {
            issue();
            umma_commit(&mbar);
        }
        ok = __syncthreads_and(mbar_wait_timed(&mbar, phase));
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return ok;
    };
    int done_tiles = 0;
    if ((int64_t)blockIdx.x < ntiles) load_row(blockIdx.x);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++done_tiles) {
        const int64_t row = tile * 128 + tid;
        const bool valid = row < ne;
        const float tgt = valid ? target[row] : 0.f;
        // features -> BF16 at columns 64-79 (the previous tile's gradient product has completed)
#pragma unroll
        for (int c = 0; c < 2; ++c)
            *reinterpret_cast<uint4*>(&sA[core_idx<kTA>(tid, 64 + 8 * c)]) =
                make_uint4(pack_bf16(f[2 * c].x, f[2 * c].y), pack_bf16(f[2 * c].z, f[2 * c].w),
                           pack_bf16(f[2 * c + 1].x, f[2 * c + 1].y), pack_bf16(f[2 * c + 1].z, f[2 * c + 1].w));
        if (tile + gridDim.x < ntiles) load_row(tile + gridDim.x);
        // layer 1: [X | 1] [W1; b1]
        if (!step([&] {
                umma_f16_id(tmem, umma_desc(a0 + 8 * 128, 128, kSboA), umma_desc(b10, 128, kSboB1), kId1, 0);
                umma_f16_id(tmem, umma_desc(a0 + 10 * 128, 128, kSboA), umma_desc(b10 + 256, 128, kSboB1), kId1, 1);
            }))
            break;
        uint32_t m1[2] = {0u, 0u};  // z1 > 0, one bit per hidden unit
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float v[32];
            tmem_ld32(acc_z + 32 * half, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) m1[half] |= (v[i] > 0.f ? 1u : 0u) << i;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                *reinterpret_cast<uint4*>(&sA[core_idx<kTA>(tid, 32 * half + 8 * c)]) =
                    make_uint4(relu_bf16x2(v[8 * c], v[8 * c + 1]), relu_bf16x2(v[8 * c + 2], v[8 * c + 3]),
                               relu_bf16x2(v[8 * c + 4], v[8 * c + 5]), relu_bf16x2(v[8 * c + 6], v[8 * c + 7]));
        }
        // layer 2: [H1 | X | 1] [W2; 0; b2]
        if (!step([&] {
#pragma unroll
                for (int c = 0; c < kTA / 16; ++c)
                    umma_f16_id(tmem, umma_desc(a0 + 256 * c, 128, kSboA), umma_desc(b20 + 256 * c, 128, kSboA), kId1, c > 0);
            }))
            break;
        {
            // two passes over z2 in halves (y needs all of it before delta_2): fewer live registers
            float y = b3;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float z[32];
                tmem_ld32(acc_z + 32 * half, z);
#pragma unroll
                for (int j = 0; j < 32; ++j) y = fmaf(fmaxf(z[j], 0.f), sw3[32 * half + j], y);
            }
            const float r3 = valid ? y - tgt : 0.f;
            const float d3 = 2.f * r3 * inv_n;
            sse = fmaf(r3, r3, sse);
            gb3 += d3;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float z[32];
                tmem_ld32(acc_z + 32 * half, z);
#pragma unroll
                for (int j = 0; j < 32; ++j) gw3[32 * half + j] = fmaf(fmaxf(z[j], 0.f), d3, gw3[32 * half + j]);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float d[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        d[e] = z[8 * c + e] > 0.f ? d3 * sw3[32 * half + 8 * c + e] : 0.f;
                    *reinterpret_cast<uint4*>(&sD[core_idx<kTD>(tid, 32 * half + 8 * c)]) =
                        make_uint4(pack_bf16(d[0], d[1]), pack_bf16(d[2], d[3]), pack_bf16(d[4], d[5]),
                                   pack_bf16(d[6], d[7]));
                }
            }
        }
        // delta_1 before the mask: delta_2 W2^T
        if (!step([&] {
#pragma unroll
                for (int c = 0; c < kH / 16; ++c)
                    umma_f16_id(tmem, umma_desc(d0 + 256 * c, 128, kSboD), umma_desc(bt0 + 256 * c, 128, kSboB2T), kId1, c > 0);
            }))
            break;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float v[32];
            tmem_ld32(acc_z + 32 * half, v);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float d[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) d[e] = (m1[half] >> (8 * c + e)) & 1u ? v[8 * c + e] : 0.f;
                *reinterpret_cast<uint4*>(&sD[core_idx<kTD>(tid, 64 + 32 * half + 8 * c)]) =
                    make_uint4(pack_bf16(d[0], d[1]), pack_bf16(d[2], d[3]), pack_bf16(d[4], d[5]),
                               pack_bf16(d[6], d[7]));
            }
        }
        // G += [delta_2 | delta_1]^T [H1 | X | 1]: both operands MN-major, K = the 128 rows
        const bool first = done_tiles == 0;
        if (!step([&] {
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    umma_f16_id(acc_g - lane_off, umma_desc_mn(d0 + 2 * kSboD * c, 128, kSboD),
                                umma_desc_mn(a0 + 2 * kSboA * c, 128, kSboA), kIdG, (first && c == 0) ? 0u : 1u);
            }))
            break;
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        // the group in flight (if any) completes before its operands and TMEM are released
        if (tid == 0) mbar_wait_timed(&mbar, phase ^ 1);
        tc_sync();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTColsTmem) : "memory");
        return;
    }
    // this CTA's partial gradient
    float* P = part + (size_t)blockIdx.x * (NP + 1);
    if (done_tiles > 0) {
        float g0[32], g1[32], g2[32];
        tmem_ld32(acc_g, g0);
        tmem_ld32(acc_g + 32, g1);
        tmem_ld32(acc_g + 64, g2);
        if (tid < kH) {
            const int j = tid;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                P[OFF_W2 + i * kH + j] = g0[i];
                P[OFF_W2 + (32 + i) * kH + j] = g1[i];
            }
            P[OFF_B2 + j] = g2[16];
        } else {
            const int i = tid - kH;
#pragma unroll
            for (int fi = 0; fi < kF; ++fi) P[OFF_W1 + fi * kH + i] = g2[fi];
            P[OFF_B1 + i] = g2[16];
        }
    } else {
        for (int i = tid; i < OFF_W3; i += 128) P[i] = 0.f;
    }
    // dw3, db3 and the squared errors: per-thread sums added over the CTA in thread order
    tc_sync();
    float* red = reinterpret_cast<float*>(base);  // the operand tiles are free now
#pragma unroll
    for (int j = 0; j < kH; ++j) red[tid * 68 + j] = gw3[j];
    red[tid * 68 + 64] = gb3;
    red[tid * 68 + 65] = sse;
    __syncthreads();
    if (tid < 66) {
        float s = 0.f;
        for (int r = 0; r < 128; ++r) s += red[r * 68 + tid];
        if (tid < kH) P[OFF_W3 + tid] = s;
        else if (tid == 64) P[OFF_B3] = s;
        else P[NP] = s;
    }
    tc_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTColsTmem) : "memory");
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
    int64_t step = 0;
    cudaStream_t stream = nullptr;
    int device = -1;
    int* err = nullptr;  // set by a tensor-core kernel whose completion wait ran out
};

static void mlp_free(sfg_mlp* n) {
    if (!n) return;
    SfgDeviceGuard guard(n->device);
    void* ptrs[] = {n->theta, n->m, n->v, n->grad, n->err};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, n->stream);
    delete n;
}

// gradient (and loss) of the network on [feats, targets) into n->grad
static sfg_status mlp_grad(sfg_ctx* ctx, sfg_mlp* n, const float* feats, const float* targets,
                           int64_t ne, double* loss_dev) {
    // two CTAs per SM (each holds 256 TMEM columns and about 113 KB of shared memory)
    const auto key = std::make_tuple((const void*)k_mlp_fwdbwd_tc, 128, kTrainSmem);
    if (ctx->occupancy.find(key) == ctx->occupancy.end()) {
        SFG_CUDA(ctx, cudaFuncSetAttribute(k_mlp_fwdbwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kTrainSmem));
        ctx->occupancy.emplace(key, 2);
    }
    const int grid = (int)std::min<int64_t>((ne + 127) / 128, (int64_t)ctx->num_sms * 2);
    Scratch s(ctx);
    float* part;
    SFG_TRY(s.get(&part, (size_t)grid * (NP + 1)));
    sfg_tic(ctx, "mlp_fwdbwd");
    k_mlp_fwdbwd_tc<<<grid, 128, kTrainSmem, ctx->stream>>>(n->theta, feats, targets, ne, part, n->err,
                                                             ctx->withhold_mma ? 1 : 0);
    sfg_toc(ctx);
    k_mlp_fold<<<ceil_div_u(NP + 1, 256), 256, 0, ctx->stream>>>(part, grid, ne, n->grad, loss_dev);
    ctx->launches += 2;
    SFG_LAUNCH_CHECK(ctx, "k_mlp_fwdbwd_tc");
    return SFG_OK;
}

sfg_status sfg_mlp_forward_impl(sfg_ctx* ctx, const sfg_mlp* net, const float* feats, int64_t ne,
                                float* out) {
    if (ne == 0) return SFG_OK;
    int* err = net->err;
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
    k_mlp_forward_tc<<<grid, 128, 0, ctx->stream>>>(net->theta, feats, ne, out, err,
                                                     ctx->withhold_mma ? 1 : 0);
    sfg_toc(ctx);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_mlp_forward_tc");
    return SFG_OK;
}

// Synchronise and report (then clear) a completion wait of this network's tensor-core kernels
// that ran out since the last check.
sfg_status sfg_mlp_check_impl(sfg_ctx* ctx, const sfg_mlp* net) {
    int h = 0;
    SFG_CUDA(ctx, cudaMemcpyAsync(&h, net->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SFG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (h) {
        SFG_CUDA(ctx, cudaMemsetAsync(net->err, 0, sizeof(int), ctx->stream));
        return sfg_fail(ctx, SFG_ETIMEOUT, "a tensor-core completion wait of the network ran out");
    }
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
    A((void**)&n->err, sizeof(int));
    if (st != SFG_OK) {
        mlp_free(n);
        return st;
    }
    SFG_CUDA(ctx, cudaMemsetAsync(n->err, 0, sizeof(int), ctx->stream));
    SFG_CUDA(ctx, cudaMemsetAsync(n->m, 0, 4 * NP, ctx->stream));
    SFG_CUDA(ctx, cudaMemsetAsync(n->v, 0, 4 * NP, ctx->stream));
    k_mlp_init<<<ceil_div_u(NP, 256), 256, 0, ctx->stream>>>(seed, n->theta);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_mlp_init");
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
    return SFG_OK;
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
        SFG_TRY(sfg_mlp_check_impl(ctx, net));
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
        }
    if (loss_host) {
        Scratch s(ctx);
        double* loss;
        SFG_TRY(s.get(&loss, 1));
        SFG_TRY(mlp_grad(ctx, net, feats, targets, ne, loss));
        SFG_CUDA(ctx, cudaMemcpyAsync(loss_host, loss, 8, cudaMemcpyDeviceToHost, ctx->stream));
        SFG_TRY(sfg_mlp_check_impl(ctx, net));
    }
    return SFG_OK;
}

sfg_status sfg_mlp_check(sfg_ctx* ctx, const sfg_mlp* net) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!net) return sfg_fail(ctx, SFG_EINVAL, "network is NULL");
    return sfg_mlp_check_impl(ctx, net);
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
