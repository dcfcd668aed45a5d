// Deterministic reductions: each block writes its partial sums (float64) to a slot indexed by its block
// number (block_partials), and one block per slice adds that slice's slots in a fixed order (slice_sum).
// Every order is fixed by the launch shape, so results are bitwise reproducible.
#pragma once

#include <cuda_runtime.h>

namespace dect {

template <int N>
__device__ __forceinline__ void block_partials(double (&v)[N], double* __restrict__ out) {
    __shared__ double red[N][32];
    for (int q = 0; q < N; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    const int w = threadIdx.x / 32;
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < N; ++q) red[q][w] = v[q];
    __syncthreads();
    if (threadIdx.x < N) {
        double t = 0.0;
        for (int k = 0; k < (int)blockDim.x / 32; ++k) t += red[threadIdx.x][k];
        out[N * (size_t)blockIdx.x + threadIdx.x] = t;
    }
}

// The same slots from float per-thread values: each warp adds its 32 values in float (a few ulps of the
// warp sum), the warp sums are added in float64. Keeps float64 work (slow on this GPU) off the
// per-element path of element-wise kernels.
template <int N>
__device__ __forceinline__ void block_partials(float (&v)[N], double* __restrict__ out) {
    __shared__ double redf[N][32];
    for (int q = 0; q < N; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    const int w = threadIdx.x / 32;
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < N; ++q) redf[q][w] = (double)v[q];
    __syncthreads();
    if (threadIdx.x < N) {
        double t = 0.0;
        for (int k = 0; k < (int)blockDim.x / 32; ++k) t += redf[threadIdx.x][k];
        out[N * (size_t)blockIdx.x + threadIdx.x] = t;
    }
}

// Sum of partial slots [prefix[s], prefix[s+1]) of width N, by one block (fixed order).
template <int N>
__device__ void slice_sum(const double* __restrict__ part, const int* __restrict__ prefix, int s, double (&out)[N]) {
    __shared__ double red[N][256];
    const int b0 = prefix[s], b1 = prefix[s + 1];
    double acc[N];
    for (int q = 0; q < N; ++q) acc[q] = 0.0;
    // unrolled so that several slots' loads are in flight; each thread still adds its slots in order
#pragma unroll 8
    for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x)
        for (int q = 0; q < N; ++q) acc[q] += part[N * (size_t)b + q];
    for (int q = 0; q < N; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int q = 0; q < N; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
        __syncthreads();
    }
    for (int q = 0; q < N; ++q) out[q] = red[q][0];
    __syncthreads();
}

}  // namespace dect
