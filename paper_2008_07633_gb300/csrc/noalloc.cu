// Allocation-free variant of sfg_affinity.
//
// sfg_affinity needs one FP64 row norm per node as scratch and takes it from the stream-ordered
// allocator. Some callers cannot let a library allocate device memory: applications that hand all
// device memory to their own pool and forbid other allocations, runtimes that must not change the
// device's memory footprint after start-up, or code that has to run where cudaMalloc and
// cudaMallocAsync are not permitted. sfg_affinity_noalloc serves them: its scratch is a
// file-scope device array of fixed size, so the call allocates nothing.
#include <mutex>

#include "sfg_internal.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int kMaxDevices = 64;

// Row-norm scratch shared by every call on a device. As file-scope device storage it is part of
// the module: every GPU that loads this library holds these SFG_AFFINITY_NOALLOC_MAX_N * 8 bytes
// until the process exits. In host code the name is only a host-side stand-in; kernels receive
// the device address obtained with cudaGetSymbolAddress.
__device__ __align__(256) double g_rownorm_scratch[SFG_AFFINITY_NOALLOC_MAX_N];

std::mutex g_mu;
double* g_scratch_dev[kMaxDevices] = {};

// ||X_p||^2 in FP64, increasing k, no fused multiply-add (same arithmetic as sfg_affinity).
__global__ void k_rownorm_static(int32_t n, const float* __restrict__ X, int K,
                                 double* __restrict__ nn) {
    for (int64_t p = (int64_t)blockIdx.x * kBlock + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * kBlock) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) {
            const double x = (double)X[p * K + k];
            s = __dadd_rn(s, __dmul_rn(x, x));
        }
        nn[p] = s;
    }
}

// delta_e = 1 - (X_p . X_q)^2 / (||X_p||^2 ||X_q||^2), FP64, no fused multiply-add.
__global__ void k_affinity_static(int64_t m, const int32_t* __restrict__ eu,
                                  const int32_t* __restrict__ ev, const float* __restrict__ X,
                                  int K, const double* __restrict__ nn,
                                  double* __restrict__ delta) {
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * kBlock) {
        const int64_t p = eu[e], q = ev[e];
        double dot = 0.0;
        for (int k = 0; k < K; ++k)
            dot = __dadd_rn(dot, __dmul_rn((double)X[p * K + k], (double)X[q * K + k]));
        const double den = __dmul_rn(nn[p], nn[q]);
        delta[e] = den > 0.0 ? __dsub_rn(1.0, __ddiv_rn(__dmul_rn(dot, dot), den)) : 1.0;
    }
}

}  // namespace

// Device address of the scratch array on ctx's device, looked up once per device and cached.
// sfg_ctx_create calls this with the context's device current. The lookup loads this file's
// module on that device (modules load lazily), and with it the array: doing it at context
// creation keeps every sfg_affinity_noalloc call free of that one-time allocation.
sfg_status sfg_noalloc_prepare(sfg_ctx* ctx) {
    const int dev = ctx->device;
    if (dev < 0 || dev >= kMaxDevices)
        return sfg_fail(ctx, SFG_EUNSUPPORTED, "device %d beyond the supported %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_rownorm_scratch);
        if (e != cudaSuccess) return sfg_cuda_fail(ctx, e, "cudaGetSymbolAddress(scratch)");
        g_scratch_dev[dev] = static_cast<double*>(p);
    }
    return SFG_OK;
}

namespace {

sfg_status scratch_address(sfg_ctx* ctx, double** out) {
    SFG_TRY(sfg_noalloc_prepare(ctx));
    std::lock_guard<std::mutex> lock(g_mu);
    *out = g_scratch_dev[ctx->device];
    return SFG_OK;
}

}  // namespace

extern "C" sfg_status sfg_affinity_noalloc(sfg_ctx* ctx, const sfg_graph* L, const float* X, int K,
                                           double* delta_out) {
    if (!ctx) return SFG_EINVAL;
    SFG_DEVICE(ctx);
    if (!L) return sfg_fail(ctx, SFG_EINVAL, "graph is NULL");
    if (K < 1) return sfg_fail(ctx, SFG_EINVAL, "K must be >= 1");
    if (L->n > SFG_AFFINITY_NOALLOC_MAX_N)
        return sfg_fail(ctx, SFG_ECAPACITY,
                        "sfg_affinity_noalloc: n = %d exceeds the fixed scratch of %d nodes "
                        "(use sfg_affinity)", L->n, SFG_AFFINITY_NOALLOC_MAX_N);
    SFG_TRY(sfg_check_dev(ctx, X, "X"));
    if (L->m > 0) SFG_TRY(sfg_check_dev(ctx, delta_out, "delta_out"));
    double* nn = nullptr;
    SFG_TRY(scratch_address(ctx, &nn));
    // every entry of nn[0, n) is rewritten below before it is read: nothing needs clearing
    k_rownorm_static<<<sfg_grid(ctx, (const void*)k_rownorm_static, kBlock, 0, L->n), kBlock, 0,
                       ctx->stream>>>(L->n, X, K, nn);
    ++ctx->launches;
    SFG_LAUNCH_CHECK(ctx, "k_rownorm_static");
    if (L->m > 0) {
        k_affinity_static<<<sfg_grid(ctx, (const void*)k_affinity_static, kBlock, 0, L->m), kBlock,
                            0, ctx->stream>>>(L->m, L->eu, L->ev, X, K, nn, delta_out);
        ++ctx->launches;
        SFG_LAUNCH_CHECK(ctx, "k_affinity_static");
    }
    return SFG_OK;
}
