// Fixed-order block sums with FP64-level accuracy in FP32 arithmetic.
//
// Partial sums are carried as unevaluated pairs hi + lo of floats and combined
// with the error-free two-sum of Knuth (s = a + b exactly equals hi + lo with
// hi = fl(a + b)), so adding n non-negative terms loses about n * 2^-44 relative
// instead of n * 2^-24: as accurate as summing the same FP32 terms in FP64, without
// the FP64 pipe, which is narrow on this GPU and made the old per-block FP64
// reductions a long serial latency chain.  The order of additions is fixed, so
// results are bitwise reproducible.
#pragma once
#include <cuda_runtime.h>

namespace elf {

struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  const float e = (a - (s - bp)) + (b - bp);
  return {s, e};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const FF s = ff_two_sum(a.hi, b.hi);
  const float e = s.lo + (a.lo + b.lo);
  const float hi = s.hi + e;
  return {hi, e - (hi - s.hi)};
}

__device__ __forceinline__ FF warp_sum_ff(FF v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const FF o = {__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off)};
    v = ff_add(v, o);
  }
  return v;
}

// Sums of NV per-thread values (floats, or pairs) over a block of whole warps (at most 32 warps, 1D or
// 2D); red holds 2 * NV floats per warp.  The results are valid in the block's first
// thread.  Contains two block barriers; every thread of the block must call it.
template <int NV>
__device__ __forceinline__ void block_sum_ff(const FF (&v)[NV], float* red, double (&out)[NV]) {
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int w = t >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
  FF s[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) s[i] = warp_sum_ff(v[i]);
  __syncthreads();  // red may still be in use by a previous call
  if ((t & 31) == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      red[(2 * NV) * w + 2 * i] = s[i].hi;
      red[(2 * NV) * w + 2 * i + 1] = s[i].lo;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) out[i] = 0.0;
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      FF x = {0.f, 0.f};
      if (t < nw) x = FF{red[(2 * NV) * t + 2 * i], red[(2 * NV) * t + 2 * i + 1]};
      x = warp_sum_ff(x);
      out[i] = (double)x.hi + (double)x.lo;
    }
  }
}

template <int NV>
__device__ __forceinline__ void block_sum_ff(const float (&v)[NV], float* red, double (&out)[NV]) {
  FF f[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) f[i] = FF{v[i], 0.f};
  block_sum_ff<NV>(f, red, out);
}

// A double as an unevaluated pair of floats (48 significant bits).
__device__ __forceinline__ FF ff_from_double(double d) {
  const float hi = (float)d;
  return {hi, (float)(d - (double)hi)};
}

}  // namespace elf
