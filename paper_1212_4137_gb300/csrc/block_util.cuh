// block_util.cuh -- deterministic block-wide reductions and scans (fixed order, no atomics),
// so that a start's result does not depend on scheduling or on the other starts.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace spca {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned warp_max_u(unsigned v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the block; every thread gets the total.  red must hold >= 32 doubles.
// The warp sums are added in warp order, so the result is the same on every run.
__device__ __forceinline__ double block_sum_d(double v, double *red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < nw; ++k) t += red[k];
  return t;
}

// FP32 sum over the block in a fixed order; every thread gets the total
__device__ __forceinline__ float block_sum_f(float v, float *red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum_f(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float t = 0.0f;
  for (int k = 0; k < nw; ++k) t += red[k];
  return t;
}

__device__ __forceinline__ int block_sum_i(int v, int *red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum_i(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  int t = 0;
  for (int k = 0; k < nw; ++k) t += red[k];
  return t;
}

__device__ __forceinline__ unsigned block_max_u(unsigned v, unsigned *red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_max_u(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  unsigned t = 0;
  for (int k = 0; k < nw; ++k) t = max(t, red[k]);
  return t;
}

// Exclusive prefix count of `flag` over the block in thread order; *total gets the count.
// All threads of the block must call it.  red must hold >= 32 ints.
__device__ __forceinline__ int block_excl_scan_flag(bool flag, int *red, int *total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const unsigned ballot = __ballot_sync(0xffffffffu, flag);
  const int in_warp = __popc(ballot & ((1u << lane) - 1u));
  __syncthreads();
  if (lane == 0) red[w] = __popc(ballot);
  __syncthreads();
  int off = 0, tot = 0;
  for (int k = 0; k < nw; ++k) {
    const int t = red[k];
    off += (k < w) ? t : 0;
    tot += t;
  }
  *total = tot;
  return off + in_warp;
}

// Compensated dot product in FP32 pairs (Ogita, Rump, Oishi 2005, "Dot2"): each product is
// split exactly into its rounded value and its error (one FMA), the running sum is kept as an
// unevaluated pair hi + lo with Knuth's two-sum, and the errors are collected in lo.  The result
// is as accurate as an FP32 sum carried in twice the precision, on the FP32 pipe (GB300 runs FP64
// at a small fraction of the FP32 rate).  The _rn intrinsics are never fused or reassociated.
struct F32Pair {
  float hi = 0.0f, lo = 0.0f;
};
__device__ __forceinline__ void f32pair_fma(F32Pair &s, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);
  const float t = __fadd_rn(s.hi, p);
  const float bv = __fsub_rn(t, s.hi);
  const float te = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bv)), __fsub_rn(p, bv));
  s.hi = t;
  s.lo = __fadd_rn(s.lo, __fadd_rn(te, pe));
}
__device__ __forceinline__ double f32pair_value(const F32Pair &s) { return (double)s.hi + (double)s.lo; }

// order-preserving key of |v|: the IEEE bits without the sign (monotone for |v| >= 0)
__device__ __forceinline__ uint32_t abs_key(float v) { return __float_as_uint(v) & 0x7fffffffu; }

}  // namespace spca
