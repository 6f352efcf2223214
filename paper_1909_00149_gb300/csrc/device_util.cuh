// Small device helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>

#include "otprox_internal.cuh"

namespace otp {

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void stg4v(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float& f4(float4& v, int e) { return (&v.x)[e]; }
__device__ __forceinline__ float f4c(const float4& v, int e) { return (&v.x)[e]; }

// Sum kNumSums per-thread FP32 partials over a block of NT threads and write
// the FP64 totals to out[0..kNumSums).  FP32 inside a warp, FP64 across warps
// (FP64 throughput is scarce on this GPU).  Must be reached by every thread.
template <int NT>
__device__ __forceinline__ void block_sums_to(float (&v)[kNumSums], double* out) {
  constexpr int NW = NT / 32;
  __shared__ double red[NW][kNumSums];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int k = 0; k < kNumSums; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kNumSums; ++k) red[warp][k] = (double)v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < kNumSums; ++k) {
      double t = lane < NW ? red[lane][k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) out[k] = t;
    }
  }
}

}  // namespace otp
