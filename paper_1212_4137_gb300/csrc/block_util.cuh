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
// integer reductions in one warp-wide instruction (redux.sync, sm_80+); exact
__device__ __forceinline__ int warp_sum_i(int v) { return __reduce_add_sync(0xffffffffu, v); }
__device__ __forceinline__ unsigned warp_max_u(unsigned v) { return __reduce_max_sync(0xffffffffu, v); }

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
// |a| of a pair (exact)
__device__ __forceinline__ F32Pair f32pair_abs(const F32Pair &a) {
  F32Pair r;
  r.hi = fabsf(a.hi);
  r.lo = a.hi < 0.0f ? -a.lo : a.lo;
  return r;
}
// a^2 of a pair: the exact square of the leading part (one FMA for its error) plus 2 hi lo,
// renormalised; relative error about 2^-44
__device__ __forceinline__ F32Pair f32pair_sq(const F32Pair &a) {
  const float p = __fmul_rn(a.hi, a.hi);
  const float e = __fadd_rn(__fmaf_rn(a.hi, a.hi, -p), __fmul_rn(__fmul_rn(2.0f, a.hi), a.lo));
  F32Pair r;
  r.hi = __fadd_rn(p, e);
  r.lo = __fsub_rn(e, __fsub_rn(r.hi, p));
  return r;
}
// a + b of two pairs: Knuth's two-sum of the leading parts (exact), the trailing parts added to
// its error, then renormalised (Dekker's fast two-sum); the same bits for a + b and b + a
__device__ __forceinline__ F32Pair f32pair_add(const F32Pair &a, const F32Pair &b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bv = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
  const float lo = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  F32Pair r;
  r.hi = __fadd_rn(s, lo);
  r.lo = __fsub_rn(lo, __fsub_rn(r.hi, s));
  return r;
}

// order-preserving key of |v|: the IEEE bits without the sign (monotone for |v| >= 0)
__device__ __forceinline__ uint32_t abs_key(float v) { return __float_as_uint(v) & 0x7fffffffu; }

}  // namespace spca
