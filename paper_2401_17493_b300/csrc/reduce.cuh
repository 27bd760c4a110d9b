// Warp- and block-level FP64 reductions shared by the kernels (deterministic:
// fixed shuffle tree, fixed warp order).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

namespace claire {

// max that keeps a NaN (fmax would drop it): the infinity norm must expose non-finite fields
__device__ __forceinline__ double nanmax(double a, double b) {
  return a != a ? a : (b != b ? b : fmax(a, b));
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double nanmin(double a, double b) {
  return a != a ? a : (b != b ? b : fmin(a, b));
}

// Reduction modes (ReduceMode): 0 sum a b, 1 sum (a - b)^2, 2 max |a|, 3 sum a^2,
// 4 max a, 5 min a, 6 sum a.  Max / min keep NaNs so non-finite fields show.
__device__ __forceinline__ bool red_is_max(int mode) { return mode == 2 || mode == 4; }
__device__ __forceinline__ double red_init(int mode) {
  return mode == 4 ? -CUDART_INF : (mode == 5 ? CUDART_INF : 0.0);
}
__device__ __forceinline__ double red_combine(int mode, double a, double b) {
  return red_is_max(mode) ? nanmax(a, b) : (mode == 5 ? nanmin(a, b) : a + b);
}
__device__ __forceinline__ double warp_red(int mode, double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = red_combine(mode, v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide reduction; the result is valid in thread (0, 0).  Works for 1D
// and 2D blocks (linear thread id); call once per kernel by every thread.
__device__ __forceinline__ double block_red(int mode, double acc) {
  __shared__ double sh[32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
  acc = warp_red(mode, acc);
  if ((tid & 31) == 0) sh[tid >> 5] = acc;
  __syncthreads();
  double v = red_init(mode);
  if (tid < 32) {
    v = tid < nwarps ? sh[tid] : red_init(mode);
    v = warp_red(mode, v);
  }
  return v;
}

__device__ __forceinline__ double block_sum(double v) { return block_red(0, v); }

// Compensated (Kahan) FP32 accumulator for per-thread partial sums: FP64
// arithmetic is slow on this part, so each thread sums its elements in FP32
// with compensation (error ~1 ulp of the partial, independent of the count)
// and only the cross-thread / cross-block reduction runs in FP64.
struct KahanF {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

}  // namespace claire
