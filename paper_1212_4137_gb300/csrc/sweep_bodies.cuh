// sweep_bodies.cuh -- the per-start bodies of the start initialisation (Algorithm 2, "select
// initial point") and of the y-step (Table 3, S1 and S2), shared by the kernels that run them one
// start per CTA: the single-problem kernels, the grouped kernels and the one-launch solve of small
// problems.
#pragma once

#include <cuda_fp16.h>

#include <cstdint>

#include "block_util.cuh"
#include "spca_internal.cuh"

namespace spca {

// ------------------------------------------------------------------ a1: start initialisation
// SplitMix64 (Steele, Lea, Flood 2014) finaliser with the published constants, used as a
// counter-based generator: word(key, i) = mix(key + (i + 1) * golden).
static __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static __device__ __forceinline__ double sm64_uniform(uint64_t key, uint64_t i) {
  return (double)(sm64_mix(key + (i + 1ull) * 0x9E3779B97F4A7C15ull) >> 11) * 0x1.0p-53;
}
// normal number i of the stream (Box-Muller over the pair i/2)
static __device__ __forceinline__ double bm_normal(uint64_t key, uint64_t i) {
  const uint64_t j = i >> 1;
  const double u1 = 1.0 - sm64_uniform(key, 2 * j), u2 = sm64_uniform(key, 2 * j + 1);
  const double rad = sqrt(-2.0 * log(u1)), ang = 6.283185307179586 * u2;
  return (i & 1) ? rad * sin(ang) : rad * cos(ang);
}

// Algorithm 2, "select initial point": x^(0) = g / ||g||_2 for the start in row c of X, taking
// start `start` (its row of x0, or normal numbers start * p + j of the seeded stream).
static __device__ void start_init_body(const float *__restrict__ x0, int64_t ld0, uint64_t key, int p,
                                       float *__restrict__ X, int64_t ldX, StartState s, double gamma0, int c,
                                       int64_t start, float *redf) {
  float *x = X + (int64_t)c * ldX;
  const float *g = x0 ? x0 + start * ld0 : nullptr;
  float part = 0.0f;
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    const float gj = g ? g[j] : (float)bm_normal(key, (uint64_t)start * (uint64_t)p + (uint64_t)j);
    x[j] = gj;
    part = fmaf(gj, gj, part);
  }
  const double nrm = sqrt((double)block_sum_f(part, redf));
  const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.0f;
  for (int j = threadIdx.x; j < p; j += blockDim.x) x[j] = x[j] * inv;
  if (threadIdx.x == 0) {
    s.status[c] = (nrm > 0.0) ? ST_ACTIVE : SPCA_ST_DEGENERATE;
    s.iters[c] = 0;
    s.nnz[c] = (nrm > 0.0) ? p : 0;
    s.F[c] = 0.0;
    s.F_prev[c] = 0.0;
    s.gamma[c] = gamma0;
    s.thr[c] = 0.0f;
    if (s.tprev) s.tprev[c] = 0.0f;
  }
}

// ------------------------------------------------------------------ y-step (Table 3 S1, S2)
// Counts the sweep for every active start; L1 variance: y = sgn(u) with sgn(0) = +1;
// L2 variance: y = u / ||u||_2, and ||u||_2 = 0 ends the start as degenerate (x = 0).
// y goes to Y (FP32) and/or to the FP16 planes of kQScale y (hi, lo; one exact plane for +-1).
static __device__ void ystep_body(int form, const float *__restrict__ U, int64_t ldu, int n,
                                  float *__restrict__ Y, __half *__restrict__ Ypl, int64_t pstride,
                                  const int *__restrict__ rank, StartState s, float *__restrict__ X, int64_t ldX,
                                  int p, int c, float *redf) {
  if (s.status[c] != ST_ACTIVE) return;
  const float *u = U + (int64_t)c * ldu;
  float *y = Y ? Y + (int64_t)c * ldu : nullptr;
  __half *yp = Ypl ? Ypl + (int64_t)(rank ? rank[c] : c) * ldu : nullptr;
  if (threadIdx.x == 0) s.iters[c] += 1;
  // four consecutive entries per thread and step (rows are 16-byte aligned: ldu is a multiple of 8)
  const int n4 = n & ~3;
  if (is_l1_var(form)) {
    for (int i = 4 * threadIdx.x; i < n4; i += 4 * blockDim.x) {
      const float4 uv = *reinterpret_cast<const float4 *>(u + i);
      const float4 yv = make_float4(uv.x >= 0.0f ? 1.0f : -1.0f, uv.y >= 0.0f ? 1.0f : -1.0f,
                                    uv.z >= 0.0f ? 1.0f : -1.0f, uv.w >= 0.0f ? 1.0f : -1.0f);
      if (y) *reinterpret_cast<float4 *>(y + i) = yv;
      if (yp) {
        // +-2^14, exact
        __half2 *h2 = reinterpret_cast<__half2 *>(yp + i);
        h2[0] = __floats2half2_rn(yv.x * kQScale, yv.y * kQScale);
        h2[1] = __floats2half2_rn(yv.z * kQScale, yv.w * kQScale);
      }
    }
    for (int i = n4 + threadIdx.x; i < n; i += blockDim.x) {
      const float yi = (u[i] >= 0.0f) ? 1.0f : -1.0f;
      if (y) y[i] = yi;
      if (yp) yp[i] = __float2half_rn(yi * kQScale);
    }
    return;
  }
  float part = 0.0f;
  for (int i = 4 * threadIdx.x; i < n4; i += 4 * blockDim.x) {
    const float4 uv = *reinterpret_cast<const float4 *>(u + i);
    part = fmaf(uv.x, uv.x, part);
    part = fmaf(uv.y, uv.y, part);
    part = fmaf(uv.z, uv.z, part);
    part = fmaf(uv.w, uv.w, part);
  }
  for (int i = n4 + threadIdx.x; i < n; i += blockDim.x) part = fmaf(u[i], u[i], part);
  const double nrm = sqrt((double)block_sum_f(part, redf));
  if (nrm == 0.0) {
    float *x = X + (int64_t)c * ldX;
    for (int j = threadIdx.x; j < p; j += blockDim.x) x[j] = 0.0f;
    if (threadIdx.x == 0) {
      s.status[c] = SPCA_ST_DEGENERATE;
      s.nnz[c] = 0;
      s.F[c] = 0.0;
    }
    return;
  }
  const float inv = (float)(1.0 / nrm);
  // y = u / ||u||_2, and its planes: kQScale y is exact (a power of two), |kQScale y| <= 2^14
  auto planes = [&](float yi, __half &hi, __half &lo) {
    const float ys = yi * kQScale;
    hi = __float2half_rn(ys);
    lo = __float2half_rn(ys - __half2float(hi));
  };
  for (int i = 4 * threadIdx.x; i < n4; i += 4 * blockDim.x) {
    const float4 uv = *reinterpret_cast<const float4 *>(u + i);
    const float4 yv = make_float4(uv.x * inv, uv.y * inv, uv.z * inv, uv.w * inv);
    if (y) *reinterpret_cast<float4 *>(y + i) = yv;
    if (yp) {
      __half h[4], l[4];
      planes(yv.x, h[0], l[0]);
      planes(yv.y, h[1], l[1]);
      planes(yv.z, h[2], l[2]);
      planes(yv.w, h[3], l[3]);
      __half2 *ph = reinterpret_cast<__half2 *>(yp + i);
      __half2 *pl = reinterpret_cast<__half2 *>(yp + pstride + i);
      ph[0] = __halves2half2(h[0], h[1]);
      ph[1] = __halves2half2(h[2], h[3]);
      pl[0] = __halves2half2(l[0], l[1]);
      pl[1] = __halves2half2(l[2], l[3]);
    }
  }
  for (int i = n4 + threadIdx.x; i < n; i += blockDim.x) {
    const float yi = u[i] * inv;
    if (y) y[i] = yi;
    if (yp) {
      __half hi, lo;
      planes(yi, hi, lo);
      yp[i] = hi;
      yp[i + pstride] = lo;
    }
  }
}

}  // namespace spca
