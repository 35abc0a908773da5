// kernel_deflate.cu -- projection deflation of the handle's matrix for a further component:
// A <- A (I - z z^T), z = x / ||x||_2.  The paper computes several components (Section 1) and
// leaves the deflation scheme open; projection deflation removes the direction z from every row.
//   1. ||x||_2 in FP64 (one CTA);
//   2. w = A z, one warp per row, each lane a compensated FP32-pair dot product (the finalise
//      accumulation), lanes combined in FP64;
//   3. A[i, j] <- A[i, j] - w_i z_j in FP64, rounded once to FP32 (columns j < p only: the
//      zero pads stay zero).
// The transposed copy and the tensor-core operands are rebuilt from A by the caller.
#include <cstdint>

#include "block_util.cuh"
#include "spca_internal.cuh"

namespace spca {

namespace {
constexpr int DT = 256;
}

__global__ void __launch_bounds__(DT) k_deflate_norm(const float *__restrict__ x, int p, double *__restrict__ inv) {
  __shared__ double red[32];
  double part = 0.0;
  for (int j = threadIdx.x; j < p; j += DT) part += (double)x[j] * (double)x[j];
  const double ss = block_sum_d(part, red);
  if (threadIdx.x == 0) *inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
}

__global__ void __launch_bounds__(DT) k_deflate_w(const float *__restrict__ A, int64_t lda, int n, int p,
                                                  const float *__restrict__ x, const double *__restrict__ inv,
                                                  double *__restrict__ w) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (DT / 32) + (threadIdx.x >> 5);
  if (i >= n) return;
  const float *row = A + (int64_t)i * lda;
  F32Pair acc;
  for (int j = lane; j < p; j += 32) f32pair_fma(acc, row[j], x[j]);
  const double t = warp_sum_d(f32pair_value(acc));
  if (lane == 0) w[i] = t * *inv;
}

__global__ void __launch_bounds__(DT) k_deflate_update(float *__restrict__ A, int64_t lda, int n, int p,
                                                       const float *__restrict__ x, const double *__restrict__ inv,
                                                       const double *__restrict__ w) {
  const int64_t total = (int64_t)n * p;
  const double s = *inv;
  for (int64_t e = (int64_t)blockIdx.x * DT + threadIdx.x; e < total; e += (int64_t)gridDim.x * DT) {
    const int64_t i = e / p, j = e - i * p;
    float *a = A + i * lda + j;
    *a = (float)((double)*a - w[i] * ((double)x[j] * s));
  }
}

cudaError_t launch_deflate(float *A, int64_t lda, int n, int p, const float *x, double *inv, double *w,
                           int sms, cudaStream_t st) {
  k_deflate_norm<<<1, DT, 0, st>>>(x, p, inv);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_deflate_w<<<(n + DT / 32 - 1) / (DT / 32), DT, 0, st>>>(A, lda, n, p, x, inv, w);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_deflate_update<<<sms > 0 ? 8 * sms : 1024, DT, 0, st>>>(A, lda, n, p, x, inv, w);
  return cudaGetLastError();
}

}  // namespace spca
