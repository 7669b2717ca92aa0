// 16-byte vector I/O for the row-major N x K block: FP32 (4 per vector) or BF16 (8 per vector),
// always widened to FP32 registers. One row of K entries is covered by LPR = K / E lanes.
#pragma once
#include <cuda_bf16.h>

template <typename T>
struct Vec;

template <>
struct Vec<float> {
    static constexpr int E = 4;
    __device__ __forceinline__ static void load(const float* p, float (&x)[4]) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
    __device__ __forceinline__ static void store(float* p, const float (&x)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    }
    // value as stored (identity for FP32)
    __device__ __forceinline__ static float round(float x) { return x; }
    // raw 16-byte load and a multiply-add of its widened entries
    __device__ __forceinline__ static uint4 load_raw(const float* p) {
        return *reinterpret_cast<const uint4*>(p);
    }
    __device__ __forceinline__ static void unpack(uint4 r, float (&x)[4]) {
        x[0] = __uint_as_float(r.x); x[1] = __uint_as_float(r.y);
        x[2] = __uint_as_float(r.z); x[3] = __uint_as_float(r.w);
    }
    __device__ __forceinline__ static void fma_raw(float w, uint4 r, float (&acc)[4]) {
        acc[0] = fmaf(w, __uint_as_float(r.x), acc[0]);
        acc[1] = fmaf(w, __uint_as_float(r.y), acc[1]);
        acc[2] = fmaf(w, __uint_as_float(r.z), acc[2]);
        acc[3] = fmaf(w, __uint_as_float(r.w), acc[3]);
    }
};

template <>
struct Vec<__nv_bfloat16> {
    static constexpr int E = 8;
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, float (&x)[8]) {
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            // bf16 -> fp32 is exact: the bf16 bits are the high half of the fp32 bits
            x[2 * i] = __uint_as_float(w[i] << 16);
            x[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
    __device__ __forceinline__ static void store(__nv_bfloat16* p, const float (&x)[8]) {
        unsigned w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);  // RN-even
            w[i] = *reinterpret_cast<const unsigned*>(&h);
        }
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __device__ __forceinline__ static float round(float x) {
        return __bfloat162float(__float2bfloat16_rn(x));
    }
    __device__ __forceinline__ static uint4 load_raw(const __nv_bfloat16* p) {
        return *reinterpret_cast<const uint4*>(p);
    }
    __device__ __forceinline__ static void unpack(uint4 r, float (&x)[8]) {
        const unsigned q[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            x[2 * i] = __uint_as_float(q[i] << 16);
            x[2 * i + 1] = __uint_as_float(q[i] & 0xffff0000u);
        }
    }
    __device__ __forceinline__ static void fma_raw(float w, uint4 r, float (&acc)[8]) {
        const unsigned q[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            acc[2 * i] = fmaf(w, __uint_as_float(q[i] << 16), acc[2 * i]);
            acc[2 * i + 1] = fmaf(w, __uint_as_float(q[i] & 0xffff0000u), acc[2 * i + 1]);
        }
    }
};
