// Device helpers shared by the CUDA translation units of libdiaq_gb300.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace diaq {

template <typename R> struct Amp;
template <> struct Amp<double> { using T = double2; };
template <> struct Amp<float> { using T = float2; };

template <typename R>
using amp_t = typename Amp<R>::T;

// Streaming loads/stores: every amplitude of a state is touched once per
// gate, so the lines are marked evict-first in L1/L2.
__device__ __forceinline__ double2 ld_stream(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(double2* p, double2 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(float2* p, float2 v) { __stcs(p, v); }

// Basis index of group g: the bits of g spread over the non-target bits,
// zeros on the targets (st: target bits in ascending order).
template <int K>
__device__ __forceinline__ int64_t insert_zeros(int64_t g, const int* st) {
#pragma unroll
    for (int a = 0; a < K; ++a) {
        const int s = st[a];
        const int64_t lo = g & ((int64_t(1) << s) - 1);
        g = ((g - lo) << 1) | lo;
    }
    return g;
}

__device__ __forceinline__ int64_t insert_zeros_rt(int64_t g, const int* st, int k) {
    for (int a = 0; a < k; ++a) {
        const int s = st[a];
        const int64_t lo = g & ((int64_t(1) << s) - 1);
        g = ((g - lo) << 1) | lo;
    }
    return g;
}

// acc (+)= m * v for one typed matrix entry; `first` starts a new sum so a
// single-term row (diagonal, permutation) is an exact copy or product.
// Entry types: 0 zero, 1 one, 2 real, 3 imaginary, 4 general.
template <typename R>
__device__ __forceinline__ void mac_typed(amp_t<R>& acc, bool& first, uint8_t type, R mr, R mi,
                                          amp_t<R> v) {
    if (type == 0) return;
    if (first) {
        first = false;
        if (type == 1) {
            acc = v;
        } else if (type == 2) {
            acc.x = mr * v.x;
            acc.y = mr * v.y;
        } else if (type == 3) {
            acc.x = -mi * v.y;
            acc.y = mi * v.x;
        } else {
            acc.x = mr * v.x;
            acc.x = fma(-mi, v.y, acc.x);
            acc.y = mr * v.y;
            acc.y = fma(mi, v.x, acc.y);
        }
    } else {
        if (type == 1) {
            acc.x += v.x;
            acc.y += v.y;
        } else if (type == 2) {
            acc.x = fma(mr, v.x, acc.x);
            acc.y = fma(mr, v.y, acc.y);
        } else if (type == 3) {
            acc.x = fma(-mi, v.y, acc.x);
            acc.y = fma(mi, v.x, acc.y);
        } else {
            acc.x = fma(mr, v.x, acc.x);
            acc.x = fma(-mi, v.y, acc.x);
            acc.y = fma(mr, v.y, acc.y);
            acc.y = fma(mi, v.x, acc.y);
        }
    }
}

// Per-thread running sum for the reductions. complex128 states accumulate
// in FP64. complex64 states form their products in FP32 (the state's own
// precision) and sum them with Kahan compensation in FP32, which carries
// about twice the FP32 mantissa, so the FP64 pipe (1/64 of the FP32 rate on
// this GPU) is not used per amplitude; the value joins the FP64 block sum.
template <typename R>
struct Acc;

template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    // s += a b - c d and s += a b + c d, two fused multiply-adds each
    __device__ __forceinline__ void add_cross(double a, double b, double c, double d) {
        s = fma(a, b, s);
        s = fma(-c, d, s);
    }
    __device__ __forceinline__ void add_dot(double a, double b, double c, double d) {
        s = fma(a, b, s);
        s = fma(c, d, s);
    }
    __device__ __forceinline__ double value() const { return s; }
};

template <>
struct Acc<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ void add_cross(float a, float b, float c_, float d) { add(fmaf(a, b, -c_ * d)); }
    __device__ __forceinline__ void add_dot(float a, float b, float c_, float d) { add(fmaf(a, b, c_ * d)); }
    __device__ __forceinline__ double value() const { return double(s) - double(c); }
};

// Deterministic block sum of one double per thread (fixed shuffle tree,
// then warp 0 over the per-warp sums). Returns the total in thread 0.
__device__ __forceinline__ double block_sum(double v, double* smem_warps) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) smem_warps[warp] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    double t = 0.0;
    if (warp == 0) {
        t = lane < nw ? smem_warps[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;
}

}  // namespace diaq
