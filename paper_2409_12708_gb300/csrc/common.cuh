// common.cuh -- device helpers shared by the THC-MPO kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace thc {

template <class T> struct Real;  // machine epsilon (unit roundoff) of the storage type
template <> struct Real<float> {
    static constexpr double eps = 5.960464477539063e-08;
};
template <> struct Real<double> {
    static constexpr double eps = 1.1102230246251565e-16;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of one value per thread; `red` is shared scratch of >= 32 entries.
template <class A>
__device__ __forceinline__ A block_sum(A v, A* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    A r = (threadIdx.x < nw) ? red[threadIdx.x] : A(0);
    if (wid == 0) r = warp_sum(r);
    if (threadIdx.x == 0) red[0] = r;
    __syncthreads();
    r = red[0];
    __syncthreads();
    return r;
}

// Block-wide maximum of one non-negative value per thread (NaN ignored);
// `red` is shared scratch of >= 32 entries.
__device__ __forceinline__ double block_max(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double r = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (wid == 0)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (threadIdx.x == 0) red[0] = r;
    __syncthreads();
    r = red[0];
    __syncthreads();
    return r;
}

__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }

// square root and sign transfer in the storage precision (no silent promotion)
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tcopysign(float a, float b) { return copysignf(a, b); }
__device__ __forceinline__ double tcopysign(double a, double b) { return copysign(a, b); }

// Device-side status word bits (one int per launch group, read by the host).
enum : int {
    DEV_OK = 0,
    DEV_NONCONVERGED = 1,   // Jacobi sweep budget exhausted
    DEV_NONFINITE = 2,      // NaN/Inf met in a decomposition
    DEV_SMALL_NONCONV = 4,  // small float64 eigensolver sweep budget exhausted
    DEV_TC_TIMEOUT = 8,     // a tensor-core kernel gave up waiting for its MMAs
};

}  // namespace thc
