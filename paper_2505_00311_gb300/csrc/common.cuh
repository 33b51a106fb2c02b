// common.cuh -- shared device helpers of the PDCS CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace pdcs {

constexpr int kWarp = 32;
constexpr int kBlock = 256;       // threads per block of the vector kernels
constexpr int kWarpsPerBlock = kBlock / kWarp;

// Cone kinds, same numbering as the C ABI.
enum ConeKind : int32_t { kZero = 0, kNonneg = 1, kSoc = 2, kRsoc = 3, kExp = 4 };

// Solver status words kept on the device.
enum : int32_t { kRunning = 0, kConverged = 1, kNumericError = 2, kTimeout = 3 };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum inside aligned groups of G lanes (G a power of two <= 32); result valid in every lane.
template <int G>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block reduction of NQ sums: fixed shuffle tree inside each warp,
// then warp results added in warp order by warp 0.  Every thread must call it.
// Returns the totals in thread 0 (other threads get partial values).
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], double (*smem)[kWarpsPerBlock]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = warp_sum(v[q]);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) smem[q][wid] = v[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double s = 0.0;
            for (int w = 0; w < kWarpsPerBlock; ++w) s += smem[q][w];
            v[q] = s;
        }
    }
    __syncthreads();
}

template <int NQ>
__device__ __forceinline__ void block_max(double (&v)[NQ], double (*smem)[kWarpsPerBlock]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = warp_max(v[q]);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) smem[q][wid] = v[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double s = 0.0;
            for (int w = 0; w < kWarpsPerBlock; ++w) s = fmax(s, smem[q][w]);
            v[q] = s;
        }
    }
    __syncthreads();
}

}  // namespace pdcs
