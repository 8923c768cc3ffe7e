// bz_device.cuh -- small device helpers shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bz {

template <typename T> struct C2;
template <> struct C2<double> { using type = double2; };
template <> struct C2<float> { using type = float2; };

template <typename V> __device__ __forceinline__ V cmk(decltype(V::x) a, decltype(V::x) b) {
    V r;
    r.x = a;
    r.y = b;
    return r;
}

// acc += a * b (complex)
template <typename V> __device__ __forceinline__ void cmac(V &acc, V a, V b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// Tiled half-spectrum layout: [cell / 32][mode][cell % 32].
__host__ __device__ __forceinline__ int64_t tiled_index(int64_t cell, int64_t mode, int64_t nhalf) {
    return (cell >> 5) * nhalf * 32 + mode * 32 + (cell & 31);
}

// Block-wide sum of up to 5 doubles; every thread receives the totals.
// `red` must hold 32 * 5 doubles of shared memory.
template <int K> __device__ __forceinline__ void block_sum(double (&v)[K], double *red) {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[warp * K + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w * K + k];   // same order in every thread
        v[k] = s;
    }
    __syncthreads();
}

// Velocity of flat grid index `idx` along dimension i (j_1 slowest).
__device__ __forceinline__ double grid_velocity(int64_t idx, int i, int dim, int N, double L,
                                                double dv) {
    int64_t t = idx;
    for (int q = dim - 1; q > i; --q) t /= N;
    return -L + (double)(t % N) * dv;
}

// Latch the first device-side error of a call into the library's error word.
__device__ __forceinline__ void raise_device_error(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

}  // namespace bz
