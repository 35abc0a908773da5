// kernel_finalise.cu -- after the sweeps: the Table 1 objective f(x) of every start with
// u = A x accumulated as a compensated FP32-pair dot product (about twice FP32's precision) and
// the norms of u summed in FP64, the explained variance (Section 4.1), the best start (ties:
// lower index), and y(x) and the support of the best x.
#include <cstdint>

#include "block_util.cuh"
#include "spca_internal.cuh"

namespace spca {

namespace {
constexpr int FT = 256;
}

// grid (r, ceil(n / FT)): u_i = sum_t x_{j_t} A[i, j_t] over the support (compensated FP32
// pairs); per-CTA FP64 partial sums of |u_i| and u_i^2 go to partials (fixed order later).
// Starts on x, row chunks on y: the CTAs in flight share row chunks, so a column slice used by
// several starts' supports is read from DRAM about once.  The columns of A are the rows of A^T:
// FP32 (row_inv null), or FP16 entries times their row's power-of-two inverse scale (the 16-bit
// copy of a resident handle; the scaled entry is exact in FP32).
template <typename T>
__global__ void __launch_bounds__(FT) k_fin_partial(const T *__restrict__ AT, const float *__restrict__ row_inv,
                                                    int64_t ldat, int n, const int *__restrict__ sup_idx,
                                                    const float *__restrict__ sup_val, int cap,
                                                    StartState st, float *__restrict__ U,
                                                    int64_t ldu, double *__restrict__ partials) {
  __shared__ int sidx[FT];
  __shared__ float sval[FT];
  __shared__ float sinv[FT];
  __shared__ double red[32];
  const int c = blockIdx.x;
  const int i = blockIdx.y * FT + threadIdx.x;
  const int nnz = st.nnz[c];
  const int *gi = sup_idx + (int64_t)c * cap;
  const float *gv = sup_val + (int64_t)c * cap;
  F32Pair acc2;
  for (int t0 = 0; t0 < nnz; t0 += FT) {
    __syncthreads();
    if (t0 + (int)threadIdx.x < nnz) {
      const int j = gi[t0 + threadIdx.x];
      sidx[threadIdx.x] = j;
      sval[threadIdx.x] = gv[t0 + threadIdx.x];
      sinv[threadIdx.x] = row_inv ? row_inv[j] : 1.0f;
    }
    __syncthreads();
    const int m = min(FT, nnz - t0);
    if (i < n)
      for (int t = 0; t < m; ++t) {
        const float a = static_cast<float>(AT[(int64_t)sidx[t] * ldat + i]) * sinv[t];
        f32pair_fma(acc2, sval[t], a);
      }
  }
  const double acc = f32pair_value(acc2);
  if (i < n) U[(int64_t)c * ldu + i] = (float)acc;
  const double l1 = block_sum_d(i < n ? fabs(acc) : 0.0, red);
  const double l2 = block_sum_d(i < n ? acc * acc : 0.0, red);
  if (threadIdx.x == 0) {
    double *o = partials + ((int64_t)c * gridDim.y + blockIdx.y) * 2;
    o[0] = l1;
    o[1] = l2;
  }
}

// block per start: add the partials in order, then f(x) of Table 1 and the explained variance
__global__ void __launch_bounds__(FT) k_fin_reduce(int form, const double *__restrict__ partials,
                                                   int nchunks, const float *__restrict__ sup_val,
                                                   int cap, StartState st) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  const int nnz = st.nnz[c];
  double a1 = 0.0;
  for (int t = threadIdx.x; t < nnz; t += FT) a1 += fabs((double)sup_val[(int64_t)c * cap + t]);
  const double x1 = block_sum_d(a1, red);
  if (threadIdx.x != 0) return;
  double l1 = 0.0, l2sq = 0.0;
  for (int b = 0; b < nchunks; ++b) {
    l1 += partials[((int64_t)c * nchunks + b) * 2 + 0];
    l2sq += partials[((int64_t)c * nchunks + b) * 2 + 1];
  }
  const double l2 = sqrt(l2sq), x0 = (double)nnz, g = st.gamma[c];
  double f;
  switch (form) {
    case 1: case 3: f = l2; break;
    case 2: case 4: f = l1; break;
    case 5: f = l2sq - g * x0; break;
    case 6: f = l1 * l1 - g * x0; break;
    case 7: f = l2 - g * x1; break;
    default: f = l1 - g * x1; break;
  }
  st.f[c] = f;
  st.ev[c] = is_l1_var(form) ? l1 : l2sq;
}

cudaError_t launch_finalise(int form, const float *AT, int64_t ldat, int n, int p, const float *X,
                            int64_t ldX, StartState s, int r, float *U, int64_t ldu,
                            const int *sup_idx, const float *sup_val, int cap, double *partials,
                            cudaStream_t st) {
  (void)p; (void)X; (void)ldX;
  const int nchunks = (n + FT - 1) / FT;
  if (nchunks > 65535) return cudaErrorInvalidValue;   // grid y limit: n above 16.7 million rows
  k_fin_partial<float><<<dim3((unsigned)r, (unsigned)nchunks), FT, 0, st>>>(AT, nullptr, ldat, n, sup_idx, sup_val,
                                                                             cap, s, U, ldu, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fin_reduce<<<r, FT, 0, st>>>(form, partials, nchunks, sup_val, cap, s);
  return cudaGetLastError();
}

cudaError_t launch_finalise_h(int form, const __half *AT16, const float *at_inv, int64_t ldat, int n, StartState s,
                              int r, float *U, int64_t ldu, const int *sup_idx, const float *sup_val, int cap,
                              double *partials, cudaStream_t st) {
  const int nchunks = (n + FT - 1) / FT;
  if (nchunks > 65535) return cudaErrorInvalidValue;
  k_fin_partial<__half><<<dim3((unsigned)r, (unsigned)nchunks), FT, 0, st>>>(AT16, at_inv, ldat, n, sup_idx,
                                                                              sup_val, cap, s, U, ldu, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_fin_reduce<<<r, FT, 0, st>>>(form, partials, nchunks, sup_val, cap, s);
  return cudaGetLastError();
}

// argmax over starts of f (or of the explained variance), ties to the lower index
__global__ void __launch_bounds__(1024) k_best(int use_ev, StartState st, int r, int *best) {
  __shared__ double sv[32];
  __shared__ int si[32];
  double bv = -INFINITY;
  int bi = 0x7fffffff;
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    const double val = use_ev ? st.ev[c] : st.f[c];
    if (val > bv) { bv = val; bi = c; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { sv[w] = bv; si[w] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
      if (sv[k] > bv || (sv[k] == bv && si[k] < bi)) { bv = sv[k]; bi = si[k]; }
    *best = (bi == 0x7fffffff) ? 0 : bi;
  }
}

cudaError_t launch_best(int form, int use_ev, StartState s, int r, int *best, cudaStream_t st) {
  (void)form;
  k_best<<<1, 1024, 0, st>>>(use_ev, s, r, best);
  return cudaGetLastError();
}

// y = y(x) (S2: sgn(u), S1: u / ||u||_2) of the best start, its x, and its support
__global__ void __launch_bounds__(1024) k_best_outputs(int form, const int *__restrict__ best,
                                                       const float *__restrict__ U, int64_t ldu, int n,
                                                       const float *__restrict__ X, int64_t ldX, int p,
                                                       float *__restrict__ y_out,
                                                       float *__restrict__ x_out,
                                                       int64_t *__restrict__ support_out,
                                                       int64_t *__restrict__ nnz_out) {
  __shared__ double red[32];
  __shared__ int redi[32];
  const int c = *best;
  const float *u = U + (int64_t)c * ldu;
  const float *x = X + (int64_t)c * ldX;
  if (is_l1_var(form)) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) y_out[i] = (u[i] >= 0.0f) ? 1.0f : -1.0f;
  } else {
    double part = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) part += (double)u[i] * (double)u[i];
    const double nrm = sqrt(block_sum_d(part, red));
    const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) y_out[i] = u[i] * inv;
  }
  int written = 0;
  for (int base = 0; base < p; base += blockDim.x) {
    const int j = base + threadIdx.x;
    const float xj = (j < p) ? x[j] : 0.0f;
    if (j < p) x_out[j] = xj;
    int tot;
    const int pos = written + block_excl_scan_flag(xj != 0.0f, redi, &tot);
    if (xj != 0.0f) support_out[pos] = j;
    written += tot;
  }
  if (threadIdx.x == 0) *nnz_out = written;
}

cudaError_t launch_best_outputs(int form, const int *best, const float *U, int64_t ldu, int n,
                                const float *X, int64_t ldX, int p, float *y_out, float *x_out,
                                int64_t *support_out, int64_t *nnz_out, cudaStream_t st) {
  k_best_outputs<<<1, 1024, 0, st>>>(form, best, U, ldu, n, X, ldX, p, y_out, x_out, support_out,
                                     nnz_out);
  return cudaGetLastError();
}

}  // namespace spca
