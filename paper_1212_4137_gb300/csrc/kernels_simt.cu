// kernels_simt.cu -- layout preparation, start initialisation, the y-step, and the FP32
// CUDA-core contractions of one AM sweep (Algorithm 2): u = A x (dense or over the support of
// x) and v = A^T y.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstdint>

#include "block_util.cuh"
#include "spca_internal.cuh"
#include "sweep_bodies.cuh"

namespace spca {

// ------------------------------------------------------------------ layout preparation
__global__ void k_transpose_f32(const float *__restrict__ src, int64_t rows, int64_t cols,
                                int64_t lds, float *__restrict__ dst, int64_t ldd) {
  __shared__ float tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  // row blocks of 32 on grid y, strided: rows may exceed 32 x 65535 (the grid's y limit)
  for (int64_t r0 = (int64_t)blockIdx.y * 32; r0 < rows; r0 += (int64_t)gridDim.y * 32) {
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
      const int64_t r = r0 + k, c = c0 + threadIdx.x;
      tile[k][threadIdx.x] = (r < rows && c < cols) ? src[r * lds + c] : 0.0f;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
      const int64_t c = c0 + k, r = r0 + threadIdx.x;  // dst row = src column
      if (c < cols && r < rows) dst[c * ldd + r] = tile[threadIdx.x][k];
    }
    __syncthreads();
  }
}

cudaError_t launch_transpose_f32(const float *src, int64_t rows, int64_t cols, int64_t lds,
                                 float *dst, int64_t ldd, cudaStream_t st) {
  const int64_t rb = (rows + 31) / 32;
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)(rb < 65535 ? rb : 65535));
  k_transpose_f32<<<grid, dim3(32, 8), 0, st>>>(src, rows, cols, lds, dst, ldd);
  return cudaGetLastError();
}

__global__ void k_convert_f64_f32(const double *__restrict__ src, int64_t rows, int64_t cols,
                                  int64_t lds, float *__restrict__ dst, int64_t ldd) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e - r * cols;
    dst[r * ldd + c] = (float)src[r * lds + c];
  }
}

cudaError_t launch_convert_f64_f32(const double *src, int64_t rows, int64_t cols, int64_t lds,
                                   float *dst, int64_t ldd, cudaStream_t st) {
  k_convert_f64_f32<<<1216, 256, 0, st>>>(src, rows, cols, lds, dst, ldd);
  return cudaGetLastError();
}

__global__ void k_copy_f32(const float *__restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                           float *__restrict__ dst, int64_t ldd) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e - r * cols;
    dst[r * ldd + c] = src[r * lds + c];
  }
}

cudaError_t launch_copy_f32(const float *src, int64_t rows, int64_t cols, int64_t lds, float *dst,
                            int64_t ldd, cudaStream_t st) {
  k_copy_f32<<<1216, 256, 0, st>>>(src, rows, cols, lds, dst, ldd);
  return cudaGetLastError();
}

__global__ void k_check_finite(const float *__restrict__ a, int64_t rows, int64_t cols, int64_t ld,
                               int *flag) {
  const int64_t total = rows * cols;
  int bad = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e - r * cols;
    bad |= !isfinite(a[r * ld + c]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

cudaError_t launch_check_finite(const float *a, int64_t rows, int64_t cols, int64_t ld, int *flag,
                                cudaStream_t st) {
  k_check_finite<<<1216, 256, 0, st>>>(a, rows, cols, ld, flag);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ a1: start initialisation
// (start_init_body: sweep_bodies.cuh)
// block per start (or per listed slot)
__global__ void __launch_bounds__(256) k_start_init(const float *__restrict__ x0, int64_t ld0,
                                                    uint64_t key, int p, float *__restrict__ X,
                                                    int64_t ldX, StartState s, double gamma0,
                                                    const int *__restrict__ slot_list,
                                                    const int *__restrict__ slot_start,
                                                    const int *__restrict__ count) {
  __shared__ float redf[32];
  if (slot_list && (int)blockIdx.x >= *count) return;
  const int c = slot_list ? slot_list[blockIdx.x] : (int)blockIdx.x;   // the slot (row of X)
  const int64_t start = slot_list ? slot_start[c] : c;                 // the start it takes
  start_init_body(x0, ld0, key, p, X, ldX, s, gamma0, c, start, redf);
}

cudaError_t launch_start_init(const float *x0, int64_t ld0, uint64_t seed, int r, int p, float *X,
                              int64_t ldX, StartState s, double gamma0, const int *slot_list,
                              const int *slot_start, const int *count, cudaStream_t st) {
  // key = mix(seed ^ mix(stream)), stream 5 = starts (same definition as the host generator)
  auto mixh = [](uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  const uint64_t key = mixh(seed ^ mixh(5ull));
  k_start_init<<<r, 256, 0, st>>>(x0, ld0, key, p, X, ldX, s, gamma0, slot_list, slot_start, count);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ y-step (Table 3 S1, S2)
// (ystep_body: sweep_bodies.cuh)
__global__ void __launch_bounds__(256) k_ystep(int form, const float *__restrict__ U, int64_t ldu,
                                               int n, float *__restrict__ Y,
                                               __half *__restrict__ Ypl, int64_t pstride,
                                               const int *__restrict__ rank, StartState s,
                                               float *__restrict__ X, int64_t ldX, int p) {
  __shared__ float redf[32];
  ystep_body(form, U, ldu, n, Y, Ypl, pstride, rank, s, X, ldX, p, (int)blockIdx.x, redf);
}

// The same for long u (n > 2 kYChunk), where one CTA per start would be latency-bound: a CTA per
// chunk of kYChunk entries and start; L2 variance first sums u_i^2 per chunk (k_ystep_norm), then
// every CTA of the start adds the chunk sums in chunk order and writes its chunk of y.
__global__ void __launch_bounds__(256) k_ystep_norm(const float *__restrict__ U, int64_t ldu, int n, StartState s,
                                                    float *__restrict__ ysum) {
  __shared__ float redf[32];
  const int b = blockIdx.x, c = blockIdx.y;
  if (s.status[c] != ST_ACTIVE) return;
  const float *u = U + (int64_t)c * ldu;
  const int i1 = min(n, (b + 1) * kYChunk);
  float part = 0.0f;
  for (int i = b * kYChunk + threadIdx.x; i < i1; i += blockDim.x) part = fmaf(u[i], u[i], part);
  const float t = block_sum_f(part, redf);
  if (threadIdx.x == 0) ysum[(int64_t)c * gridDim.x + b] = t;
}

__global__ void __launch_bounds__(256) k_ystep_apply(int form, const float *__restrict__ U, int64_t ldu, int n,
                                                     float *__restrict__ Y, __half *__restrict__ Ypl,
                                                     int64_t pstride, const int *__restrict__ rank, StartState s,
                                                     float *__restrict__ X, int64_t ldX, int p,
                                                     const float *__restrict__ ysum) {
  const int b = blockIdx.x, c = blockIdx.y, nch = gridDim.x;
  // (the chunk-0 CTA alone may change the status below, and only when every CTA of the start
  // returns without writing: ||u||_2 = 0)
  if (s.status[c] != ST_ACTIVE) return;
  const float *u = U + (int64_t)c * ldu;
  float *y = Y ? Y + (int64_t)c * ldu : nullptr;
  __half *yp = Ypl ? Ypl + (int64_t)(rank ? rank[c] : c) * ldu : nullptr;
  const int i1 = min(n, (b + 1) * kYChunk);
  if (b == 0 && threadIdx.x == 0) s.iters[c] += 1;
  if (is_l1_var(form)) {
    for (int i = b * kYChunk + threadIdx.x; i < i1; i += blockDim.x) {
      const float yi = (u[i] >= 0.0f) ? 1.0f : -1.0f;
      if (y) y[i] = yi;
      if (yp) yp[i] = __float2half_rn(yi * kQScale);
    }
    return;
  }
  float tot = 0.0f;
  for (int q = 0; q < nch; ++q) tot += ysum[(int64_t)c * nch + q];
  const double nrm = sqrt((double)tot);
  if (nrm == 0.0) {
    if (b == 0) {
      float *x = X + (int64_t)c * ldX;
      for (int j = threadIdx.x; j < p; j += blockDim.x) x[j] = 0.0f;
      if (threadIdx.x == 0) {
        s.status[c] = SPCA_ST_DEGENERATE;
        s.nnz[c] = 0;
        s.F[c] = 0.0;
      }
    }
    return;
  }
  const float inv = (float)(1.0 / nrm);
  for (int i = b * kYChunk + threadIdx.x; i < i1; i += blockDim.x) {
    const float yi = u[i] * inv;
    if (y) y[i] = yi;
    if (yp) {
      const float ys = yi * kQScale;
      const __half hi = __float2half_rn(ys);
      yp[i] = hi;
      yp[i + pstride] = __float2half_rn(ys - __half2float(hi));
    }
  }
}

cudaError_t launch_ystep(int form, const float *U, int64_t ldu, int n, int r, float *Y, void *Ypl,
                         int64_t plane_stride, const int *rank, StartState s, float *X, int64_t ldX,
                         int p, float *ysum, cudaStream_t st) {
  const int nch = (n + kYChunk - 1) / kYChunk;
  if (ysum && nch > 2) {
    const dim3 grid((unsigned)nch, (unsigned)r);
    if (!is_l1_var(form)) {
      k_ystep_norm<<<grid, 256, 0, st>>>(U, ldu, n, s, ysum);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    k_ystep_apply<<<grid, 256, 0, st>>>(form, U, ldu, n, Y, static_cast<__half *>(Ypl), plane_stride, rank, s, X,
                                        ldX, p, ysum);
    return cudaGetLastError();
  }
  k_ystep<<<r, 256, 0, st>>>(form, U, ldu, n, Y, static_cast<__half *>(Ypl), plane_stride, rank,
                             s, X, ldX, p);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ active-start list
// one CTA: ordered compaction of the flags status[c] == ST_ACTIVE over r starts
__device__ void active_list_body(const int *__restrict__ status, const int *__restrict__ nnz, int r,
                                 int *__restrict__ act, int *__restrict__ rank, Ctrl *__restrict__ ctrl) {
  __shared__ int red[32];
  __shared__ long long red_l[32];
  __shared__ int red_m[32];
  int base_pos = 0;
  long long nz = 0;
  int mz = 0;
  for (int base = 0; base < r; base += blockDim.x) {
    const int c = base + threadIdx.x;
    const bool on = c < r && status[c] == ST_ACTIVE;
    int tot;
    const int pos = base_pos + block_excl_scan_flag(on, red, &tot);
    if (on) {
      act[pos] = c;
      rank[c] = pos;
      if (nnz) {
        nz += nnz[c];
        mz = max(mz, nnz[c]);
      }
    }
    base_pos += tot;
  }
  // sum of the active support sizes (a bound on the size of their union)
  for (int o = 16; o > 0; o >>= 1) {
    nz += __shfl_xor_sync(0xffffffffu, nz, o);
    mz = max(mz, __shfl_xor_sync(0xffffffffu, mz, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red_l[threadIdx.x >> 5] = nz;
    red_m[threadIdx.x >> 5] = mz;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    int m = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      t += red_l[k];
      m = max(m, red_m[k]);
    }
    ctrl->max_nnz = m;
    ctrl->active = base_pos;
    ctrl->use_gather = (ctrl->need_dense == 0 && base_pos > 0) ? 1 : 0;
    ctrl->sum_nnz = (int)(t < 0x7fffffffLL ? t : 0x7fffffffLL);
  }
}

__global__ void __launch_bounds__(1024) k_active_list(const int *__restrict__ status, const int *__restrict__ nnz,
                                                      int r, int *__restrict__ act, int *__restrict__ rank,
                                                      Ctrl *__restrict__ ctrl) {
  active_list_body(status, nnz, r, act, rank, ctrl);
}

cudaError_t launch_active_list(const int *status, const int *nnz, int r, int *act, int *rank, Ctrl *c,
                               cudaStream_t st) {
  k_active_list<<<1, 1024, 0, st>>>(status, nnz, r, act, rank, c);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ FP32 CUDA-core GEMM
// C[m, j] = sum_k P[m, k] Q[j, k]; P (M x K) and Q (N x K) are both K-contiguous with
// leading dimensions that are multiples of 8 and zero pads, and K is a multiple of 8.
// 128 x 128 tile, 8-deep K slices, 256 threads with an 8 x 8 register block each; the
// next slice is prefetched into registers while the current one is multiplied.
namespace {
constexpr int BM = 128, BN = 128, BK = 8;
}

__global__ void __launch_bounds__(256) k_gemm_nt_f32(const float *__restrict__ P, int64_t ldp,
                                                     const float *__restrict__ Q, int64_t ldq,
                                                     float *__restrict__ C, int64_t ldc, int M,
                                                     int N, int K, const int *__restrict__ gate) {
  if (gate && *gate == 0) return;
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  // loader: thread -> (row, 4 consecutive k)
  const int lrow = tid >> 1, lk = (tid & 1) * 4;
  const bool pa = (m0 + lrow) < M, qa = (n0 + lrow) < N;
  const float *pp = P + (int64_t)(pa ? m0 + lrow : 0) * ldp + lk;
  const float *qp = Q + (int64_t)(qa ? n0 + lrow : 0) * ldq + lk;
  // compute: thread -> rows {ty*4..+3, 64+ty*4..+3}, cols {tx*4..+3, 64+tx*4..+3}
  const int ty = tid >> 4, tx = tid & 15;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

  float4 ra = pa ? *reinterpret_cast<const float4 *>(pp) : make_float4(0, 0, 0, 0);
  float4 rb = qa ? *reinterpret_cast<const float4 *>(qp) : make_float4(0, 0, 0, 0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    __syncthreads();
    As[lk + 0][lrow] = ra.x; As[lk + 1][lrow] = ra.y; As[lk + 2][lrow] = ra.z; As[lk + 3][lrow] = ra.w;
    Bs[lk + 0][lrow] = rb.x; Bs[lk + 1][lrow] = rb.y; Bs[lk + 2][lrow] = rb.z; Bs[lk + 3][lrow] = rb.w;
    __syncthreads();
    if (k0 + BK < K) {
      ra = pa ? *reinterpret_cast<const float4 *>(pp + k0 + BK) : make_float4(0, 0, 0, 0);
      rb = qa ? *reinterpret_cast<const float4 *>(qp + k0 + BK) : make_float4(0, 0, 0, 0);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + ((i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int nn = n0 + ((j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (nn < N) C[(int64_t)m * ldc + nn] = acc[i][j];
    }
  }
}

cudaError_t launch_gemm_nt_f32(const float *P, int64_t ldp, const float *Q, int64_t ldq, float *C,
                               int64_t ldc, int M, int N, int K, const int *gate, cudaStream_t st) {
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
  k_gemm_nt_f32<<<grid, 256, 0, st>>>(P, ldp, Q, ldq, C, ldc, M, N, K, gate);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ u = A x over supp(x)
// U[c, i] = sum_t val[c, t] AT[idx[c, t], i] (t over the support of x, ascending index).
// Runs only when *gate != 0 (the control word chose this path for the sweep).
// Grid: x over the starts, y over row blocks of 512 (128 threads), so the CTAs in flight share a
// few row blocks: their slices of the columns in the starts' supports (512 rows x 4 bytes each;
// 37 MB per row block for 18,000 distinct columns) stay in L2, and a column used by several
// starts is read from DRAM about once.
constexpr int kGatherThreads = 128;
// rows 4 (yb kGatherThreads + t) .. + 3 of u = A x for start c (block of kGatherThreads threads)
__device__ void gather_body(const float *__restrict__ AT, int64_t ldat, int n, const int *__restrict__ sup_idx,
                            const float *__restrict__ sup_val, int cap, StartState s, float *__restrict__ U,
                            int64_t ldu, int c, int yb, int *sidx, float *sval) {
  if (s.status[c] != ST_ACTIVE) return;
  if (s.iters[c] == 0) return;   // a start not swept yet has a dense x: the dense contraction
  const int nnz = s.nnz[c];
  // four consecutive rows per thread, read as one 16-byte vector (ldat is a multiple of 8, so
  // the rows up to the padded width are in bounds); eight columns' loads are issued before
  // their FMAs, which still run in support order
  const int i4 = (yb * kGatherThreads + threadIdx.x) * 4;
  const int *gi = sup_idx + (int64_t)c * cap;
  const float *gv = sup_val + (int64_t)c * cap;
  float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  auto step = [&](float xv, float4 a) {
    acc.x = fmaf(xv, a.x, acc.x);
    acc.y = fmaf(xv, a.y, acc.y);
    acc.z = fmaf(xv, a.z, acc.z);
    acc.w = fmaf(xv, a.w, acc.w);
  };
  for (int t0 = 0; t0 < nnz; t0 += kGatherThreads) {
    __syncthreads();
    if (t0 + (int)threadIdx.x < nnz) {
      sidx[threadIdx.x] = gi[t0 + threadIdx.x];
      sval[threadIdx.x] = gv[t0 + threadIdx.x];
    }
    __syncthreads();
    const int m = min(kGatherThreads, nnz - t0);
    if (i4 < n) {
      const float *base = AT + i4;
      int t = 0;
      for (; t + 8 <= m; t += 8) {
        float4 a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = __ldg(reinterpret_cast<const float4 *>(base + (int64_t)sidx[t + q] * ldat));
#pragma unroll
        for (int q = 0; q < 8; ++q) step(sval[t + q], a[q]);
      }
      for (; t < m; ++t) step(sval[t], __ldg(reinterpret_cast<const float4 *>(base + (int64_t)sidx[t] * ldat)));
    }
  }
  float *u = U + (int64_t)c * ldu;
  if (i4 < n) u[i4] = acc.x;
  if (i4 + 1 < n) u[i4 + 1] = acc.y;
  if (i4 + 2 < n) u[i4 + 2] = acc.z;
  if (i4 + 3 < n) u[i4 + 3] = acc.w;
}

// gather_body over the leading FP16 plane of A^T (a resident 16-bit handle): row j of the plane
// is A[:, j] times its power-of-two scale, undone by folding at_inv[j] into x_j (exact); four rows
// per thread as one 8-byte load, products and sums in FP32 in support order
__device__ void gather_lowp_body(const __half *__restrict__ AT0, const float *__restrict__ at_inv, int64_t ldat,
                                 int n, const int *__restrict__ sup_idx, const float *__restrict__ sup_val, int cap,
                                 StartState s, float *__restrict__ U, int64_t ldu, int c, int yb, int *sidx,
                                 float *sval) {
  if (s.status[c] != ST_ACTIVE) return;
  if (s.iters[c] == 0) return;   // a start not swept yet has a dense x: the dense contraction
  const int nnz = s.nnz[c];
  const int i4 = (yb * kGatherThreads + threadIdx.x) * 4;
  const int *gi = sup_idx + (int64_t)c * cap;
  const float *gv = sup_val + (int64_t)c * cap;
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  auto step = [&](float xv, uint2 raw) {
    const __half2 *h2 = reinterpret_cast<const __half2 *>(&raw);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float2 f = __half22float2(h2[q]);
      acc[2 * q] = fmaf(xv, f.x, acc[2 * q]);
      acc[2 * q + 1] = fmaf(xv, f.y, acc[2 * q + 1]);
    }
  };
  for (int t0 = 0; t0 < nnz; t0 += kGatherThreads) {
    __syncthreads();
    if (t0 + (int)threadIdx.x < nnz) {
      const int j = gi[t0 + threadIdx.x];
      sidx[threadIdx.x] = j;
      sval[threadIdx.x] = gv[t0 + threadIdx.x] * at_inv[j];
    }
    __syncthreads();
    const int m = min(kGatherThreads, nnz - t0);
    if (i4 < n) {
      const __half *base = AT0 + i4;
      int t = 0;
      for (; t + 8 <= m; t += 8) {
        uint2 a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = __ldg(reinterpret_cast<const uint2 *>(base + (int64_t)sidx[t + q] * ldat));
#pragma unroll
        for (int q = 0; q < 8; ++q) step(sval[t + q], a[q]);
      }
      for (; t < m; ++t) step(sval[t], __ldg(reinterpret_cast<const uint2 *>(base + (int64_t)sidx[t] * ldat)));
    }
  }
  float *u = U + (int64_t)c * ldu;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (i4 + q < n) u[i4 + q] = acc[q];
}

// The same gather over the leading FP16 plane of A^T (the low-precision sweeps): row j of the
// plane is A[:, j] times at_scale[j]; the inverse scale is folded into x_j.  8 rows per thread as
// one 16-byte load, products and sums in FP32 in support order.
__global__ void __launch_bounds__(256) k_gemm1_sparse_lowp(const __half *__restrict__ AT0, int64_t ldat,
                                                           const float *__restrict__ at_inv, int n,
                                                           const int *__restrict__ sup_idx,
                                                           const float *__restrict__ sup_val, int cap,
                                                           StartState s, float *__restrict__ U, int64_t ldu,
                                                           const int *__restrict__ gate) {
  if (*gate == 0) return;
  const int c = blockIdx.x;
  if (s.status[c] != ST_ACTIVE) return;
  __shared__ int sidx[256];
  __shared__ float sval[256];
  const int nnz = s.nnz[c];
  const int i8 = (blockIdx.y * blockDim.x + threadIdx.x) * 8;
  const int *gi = sup_idx + (int64_t)c * cap;
  const float *gv = sup_val + (int64_t)c * cap;
  float acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
  auto step = [&](float xv, uint4 raw) {
    const __half2 *h2 = reinterpret_cast<const __half2 *>(&raw);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 f = __half22float2(h2[q]);
      acc[2 * q] = fmaf(xv, f.x, acc[2 * q]);
      acc[2 * q + 1] = fmaf(xv, f.y, acc[2 * q + 1]);
    }
  };
  for (int t0 = 0; t0 < nnz; t0 += 256) {
    __syncthreads();
    if (t0 + (int)threadIdx.x < nnz) {
      const int j = gi[t0 + threadIdx.x];
      sidx[threadIdx.x] = j;
      sval[threadIdx.x] = gv[t0 + threadIdx.x] * at_inv[j];
    }
    __syncthreads();
    const int m = min(256, nnz - t0);
    if (i8 < n) {
      const __half *base = AT0 + i8;
      int t = 0;
      for (; t + 8 <= m; t += 8) {
        uint4 a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = __ldg(reinterpret_cast<const uint4 *>(base + (int64_t)sidx[t + q] * ldat));
#pragma unroll
        for (int q = 0; q < 8; ++q) step(sval[t + q], a[q]);
      }
      for (; t < m; ++t) step(sval[t], __ldg(reinterpret_cast<const uint4 *>(base + (int64_t)sidx[t] * ldat)));
    }
  }
  float *u = U + (int64_t)c * ldu;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (i8 + q < n) u[i8 + q] = acc[q];
}

// The same gather over the FP8 E4M3 copy of A^T (the low-precision sweeps of an FP8 handle): row j
// is A[:, j] times its scale, undone with at8_inv[j] folded into x_j; 16 rows per thread as one
// 16-byte load, products and sums in FP32 in support order.
__global__ void __launch_bounds__(256) k_gemm1_sparse_f8(const uint8_t *__restrict__ AT8, int64_t ldat,
                                                         const float *__restrict__ at_inv, int n,
                                                         const int *__restrict__ sup_idx,
                                                         const float *__restrict__ sup_val, int cap, StartState s,
                                                         float *__restrict__ U, int64_t ldu,
                                                         const int *__restrict__ gate) {
  if (*gate == 0) return;
  const int c = blockIdx.x;
  if (s.status[c] != ST_ACTIVE) return;
  __shared__ int sidx[256];
  __shared__ float sval[256];
  const int nnz = s.nnz[c];
  const int i16 = (blockIdx.y * blockDim.x + threadIdx.x) * 16;
  const int *gi = sup_idx + (int64_t)c * cap;
  const float *gv = sup_val + (int64_t)c * cap;
  float acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
  auto step = [&](float xv, uint4 raw) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[q] >> (16 * h)), __NV_E4M3);
        const float2 f = __half22float2(__half2(hr));
        acc[4 * q + 2 * h] = fmaf(xv, f.x, acc[4 * q + 2 * h]);
        acc[4 * q + 2 * h + 1] = fmaf(xv, f.y, acc[4 * q + 2 * h + 1]);
      }
    }
  };
  for (int t0 = 0; t0 < nnz; t0 += 256) {
    __syncthreads();
    if (t0 + (int)threadIdx.x < nnz) {
      const int j = gi[t0 + threadIdx.x];
      sidx[threadIdx.x] = j;
      sval[threadIdx.x] = gv[t0 + threadIdx.x] * at_inv[j];
    }
    __syncthreads();
    const int m = min(256, nnz - t0);
    if (i16 < n) {
      const uint8_t *base = AT8 + i16;
      int t = 0;
      for (; t + 8 <= m; t += 8) {
        uint4 a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = __ldg(reinterpret_cast<const uint4 *>(base + (int64_t)sidx[t + q] * ldat));
#pragma unroll
        for (int q = 0; q < 8; ++q) step(sval[t + q], a[q]);
      }
      for (; t < m; ++t) step(sval[t], __ldg(reinterpret_cast<const uint4 *>(base + (int64_t)sidx[t] * ldat)));
    }
  }
  float *u = U + (int64_t)c * ldu;
#pragma unroll
  for (int q = 0; q < 16; ++q)
    if (i16 + q < n) u[i16 + q] = acc[q];
}

cudaError_t launch_gemm1_sparse_f8(const uint8_t *AT8, int64_t ldat, const float *at_inv, int n, const int *sup_idx,
                                   const float *sup_val, int cap, StartState s, int r, float *U, int64_t ldu,
                                   const int *gate, cudaStream_t st) {
  if (ldat % 16 != 0 || (reinterpret_cast<uintptr_t>(AT8) & 15u) != 0) return cudaErrorInvalidValue;
  dim3 grid((unsigned)r, (unsigned)((n + 4095) / 4096));
  k_gemm1_sparse_f8<<<grid, 256, 0, st>>>(AT8, ldat, at_inv, n, sup_idx, sup_val, cap, s, U, ldu, gate);
  return cudaGetLastError();
}

cudaError_t launch_gemm1_sparse_lowp(const void *AT0, int64_t ldat, const float *at_inv, int n, const int *sup_idx,
                                     const float *sup_val, int cap, StartState s, int r, float *U, int64_t ldu,
                                     const int *gate, cudaStream_t st) {
  if (ldat % 8 != 0 || (reinterpret_cast<uintptr_t>(AT0) & 15u) != 0) return cudaErrorInvalidValue;
  dim3 grid((unsigned)r, (unsigned)((n + 2047) / 2048));
  k_gemm1_sparse_lowp<<<grid, 256, 0, st>>>(static_cast<const __half *>(AT0), ldat, at_inv, n, sup_idx, sup_val,
                                            cap, s, U, ldu, gate);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kGatherThreads) k_gemm1_sparse(const float *__restrict__ AT, int64_t ldat,
                                                      int n, const int *__restrict__ sup_idx,
                                                      const float *__restrict__ sup_val, int cap,
                                                      StartState s, float *__restrict__ U,
                                                      int64_t ldu, const int *__restrict__ gate) {
  __shared__ int sidx[kGatherThreads];
  __shared__ float sval[kGatherThreads];
  if (*gate == 0) return;
  gather_body(AT, ldat, n, sup_idx, sup_val, cap, s, U, ldu, (int)blockIdx.x, (int)blockIdx.y, sidx, sval);
}

cudaError_t launch_gemm1_sparse(const float *AT, int64_t ldat, int n, const int *sup_idx,
                                const float *sup_val, int cap, StartState s, int r, float *U,
                                int64_t ldu, const int *gate, cudaStream_t st) {
  if (ldat % 4 != 0 || (reinterpret_cast<uintptr_t>(AT) & 15u) != 0) return cudaErrorInvalidValue;
  const int blocks = (n + 4 * kGatherThreads - 1) / (4 * kGatherThreads);
  if (blocks > 65535) return cudaErrorInvalidValue;   // grid y limit: n above 33.5 million rows
  dim3 grid((unsigned)r, (unsigned)blocks);
  k_gemm1_sparse<<<grid, kGatherThreads, 0, st>>>(AT, ldat, n, sup_idx, sup_val, cap, s, U, ldu, gate);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ groups of problems
// The per-start phases for all problems of a group in one launch each: block g (or blockIdx.x for
// the per-problem active lists) looks its problem up and runs the single-problem body on that
// problem's blocks of the workspace.
__global__ void __launch_bounds__(256) k_g_start_init(const GProb *__restrict__ P, const int *__restrict__ prob) {
  __shared__ float redf[32];
  const GProb &q = P[prob[blockIdx.x]];
  if (!q.first) return;   // only the members whose first sweep is next
  const int c = (int)blockIdx.x - q.start0;
  start_init_body(q.x0, q.ld0, q.key, q.p, q.X, q.ldX, q.st, q.gamma0, c, c, redf);
}

cudaError_t launch_g_start_init(const GProb *P, const int *prob, int R, cudaStream_t st) {
  k_g_start_init<<<R, 256, 0, st>>>(P, prob);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(1024) k_g_active(const GProb *__restrict__ P, int parity, int only_first) {
  const GProb &q = P[blockIdx.x];
  if (only_first && !q.first) return;
  active_list_body(q.st.status, q.st.nnz, q.r, q.act, q.rank, q.ctrl[parity]);
}

cudaError_t launch_g_active(const GProb *P, int np, int parity, bool only_first, cudaStream_t st) {
  k_g_active<<<np, 1024, 0, st>>>(P, parity, only_first ? 1 : 0);
  return cudaGetLastError();
}

// many small device copies in one launch (block i copies list[i]): 16 bytes at a time where both
// ends are 16-byte aligned, else byte by byte
__global__ void k_copy_list(const CopyDesc *__restrict__ list) {
  const CopyDesc d = list[blockIdx.x];
  const char *src = static_cast<const char *>(d.src);
  char *dst = static_cast<char *>(d.dst);
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
    const int64_t n16 = d.bytes / 16;
    for (int64_t i = threadIdx.x; i < n16; i += blockDim.x)
      reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(src)[i];
    for (int64_t i = 16 * n16 + threadIdx.x; i < d.bytes; i += blockDim.x) dst[i] = src[i];
  } else {
    for (int64_t i = threadIdx.x; i < d.bytes; i += blockDim.x) dst[i] = src[i];
  }
}

cudaError_t launch_copy_list(const CopyDesc *list, int count, cudaStream_t st) {
  if (count < 1) return cudaSuccess;
  k_copy_list<<<count, 256, 0, st>>>(list);
  return cudaGetLastError();
}

// the control words of one sweep parity: cleared before an x-step, and their active counts gathered
// for the host (out[i] = problem i's count)
__global__ void k_g_ctrl(const GProb *__restrict__ P, int np, int parity, int clear, int *__restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    Ctrl *c = P[i].ctrl[parity];
    if (clear) {
      *c = Ctrl{};
    } else {
      out[i] = c->active;
    }
  }
}

cudaError_t launch_g_ctrl(const GProb *P, int np, int parity, int clear, int *out, cudaStream_t st) {
  k_g_ctrl<<<(np + 255) / 256, 256, 0, st>>>(P, np, parity, clear, out);
  return cudaGetLastError();
}

// FP16 planes of x for the dense u = A x (the first sweep): per active start, the power-of-two
// scale putting max |x_j| in [2^13, 2^14), then hi = fp16(s x), lo = fp16(s x - hi) at the start's
// packed row (its rank), and 1 / s at the same index
__global__ void __launch_bounds__(256) k_g_xplanes(const GProb *__restrict__ P, const int *__restrict__ prob) {
  __shared__ unsigned red[32];
  const GProb &q = P[prob[blockIdx.x]];
  const int c = (int)blockIdx.x - q.start0;
  // only starts not swept yet (a problem's first sweep; the others take the support gather)
  if (q.st.status[c] != ST_ACTIVE || q.st.iters[c] != 0) return;
  const float *x = q.X + (int64_t)c * q.ldX;
  unsigned mk = 0u;
  for (int j = threadIdx.x; j < q.p; j += blockDim.x) mk = max(mk, __float_as_uint(fabsf(x[j])));
  const unsigned m = block_max_u(mk, red);
  int e = 0;
  if (m != 0u) e = max(-120, min(120, 13 - ilogbf(__uint_as_float(m))));
  const float sc = ldexpf(1.0f, e);
  const int row = q.rank[c];
  __half *hi = q.Xpl + (int64_t)row * q.ldX;
  for (int j = threadIdx.x; j < q.p; j += blockDim.x) {
    const float a = x[j] * sc;
    const __half h = __float2half_rn(a);
    hi[j] = h;
    hi[j + q.xps] = __float2half_rn(a - __half2float(h));
  }
  if (threadIdx.x == 0) {
    q.x_scale[row] = sc;
    q.x_inv[row] = ldexpf(1.0f, -e);
  }
}

cudaError_t launch_g_xplanes(const GProb *P, const int *prob, int R, cudaStream_t st) {
  k_g_xplanes<<<R, 256, 0, st>>>(P, prob);
  return cudaGetLastError();
}

// grid (R, row blocks of the largest n): blocks past a problem's n exit
__global__ void __launch_bounds__(kGatherThreads) k_g_gather(const GProb *__restrict__ P, const int *__restrict__ prob) {
  __shared__ int sidx[kGatherThreads];
  __shared__ float sval[kGatherThreads];
  const GProb &q = P[prob[blockIdx.x]];
  if ((int)blockIdx.y * 4 * kGatherThreads >= q.n) return;
  const int c = (int)blockIdx.x - q.start0;
  if (q.AT16)
    gather_lowp_body(q.AT16, q.at_inv, q.ldAT, q.n, q.sup_idx, q.sup_val, q.p, q.st, q.U, q.ldU, c, (int)blockIdx.y,
                     sidx, sval);
  else
    gather_body(q.AT32, q.ldAT, q.n, q.sup_idx, q.sup_val, q.p, q.st, q.U, q.ldU, c, (int)blockIdx.y, sidx, sval);
}

cudaError_t launch_g_gather(const GProb *P, const int *prob, int R, int max_n, cudaStream_t st) {
  const int blocks = (max_n + 4 * kGatherThreads - 1) / (4 * kGatherThreads);
  if (blocks > 65535 || R > 0x7fffffff) return cudaErrorInvalidValue;
  k_g_gather<<<dim3((unsigned)R, (unsigned)blocks), kGatherThreads, 0, st>>>(P, prob);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_g_ystep(const GProb *__restrict__ P, const int *__restrict__ prob) {
  __shared__ float redf[32];
  const GProb &q = P[prob[blockIdx.x]];
  const int c = (int)blockIdx.x - q.start0;
  // the member's active starts sit at its pool's Y rows *yoff + rank
  __half *ypl = q.Ypl + (q.yoff ? (int64_t)*q.yoff * q.ldU : 0);
  ystep_body(q.form, q.U, q.ldU, q.n, nullptr, ypl, q.yps, q.rank, q.st, q.X, q.ldX, q.p, c, redf);
}

__global__ void __launch_bounds__(256) k_g_pools(const GPool *__restrict__ pools, const GProb *__restrict__ P,
                                                 const int *__restrict__ members, int parity) {
  const GPool q = pools[blockIdx.x];
  if (threadIdx.x == 0) {   // Y row offsets in member order
    int acc = 0;
    for (int k = 0; k < q.nmem; ++k) {
      const GProb &m = P[members[q.first + k]];
      *m.yoff = acc;
      acc += m.ctrl[parity]->active;
    }
    *q.count = acc;
  }
  __syncthreads();   // (the offsets are this block's own global writes)
  for (int k = 0; k < q.nmem; ++k) {
    const GProb &m = P[members[q.first + k]];
    const int a = m.ctrl[parity]->active, o = *m.yoff;
    for (int t = threadIdx.x; t < a; t += blockDim.x) q.colmap[o + t] = m.vbase + m.act[t];
  }
}

cudaError_t launch_g_pools(const GPool *pools, int npool, const GProb *P, const int *members, int parity,
                           cudaStream_t st) {
  if (npool < 1) return cudaSuccess;
  k_g_pools<<<npool, 256, 0, st>>>(pools, P, members, parity);
  return cudaGetLastError();
}

cudaError_t launch_g_ystep(const GProb *P, const int *prob, int R, cudaStream_t st) {
  k_g_ystep<<<R, 256, 0, st>>>(P, prob);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ few starts: streaming GEMV
// out[orow(c)][m] = sum_k P[m, k] Q[qrow(c), k] for the first *count (<= R) starts: the Q rows in
// shared memory, a warp per row of P (two rows for R >= 4, which then share each read of Q) read
// once with 16-byte loads, each lane's R sums per row over its strided part, then the warp's
// sums in a fixed butterfly.  Q rows longer than the shared memory holds are taken in chunks of
// Kc columns (the row sums carried in registers across the chunks, in K order).
// P's rows and Q's rows are zero past K up to the next multiple of 4 (padded layouts).
template <int R, int NR>
__global__ void __launch_bounds__(512, 1) k_gemv(const float *__restrict__ P, int64_t ldp, int M, int K, int Kc,
                                                 const float *__restrict__ Q, int64_t ldq,
                                                 const int *__restrict__ rows, const int *__restrict__ count,
                                                 float *__restrict__ out, int64_t ldo, const int *__restrict__ gate) {
  extern __shared__ __align__(16) float qs[];
  if (gate && *gate == 0) return;
  const int cnt = count ? min(*count, R) : R;
  if (cnt <= 0) return;
  const int K4 = (K + 3) / 4, Kp = 4 * K4;
  const int nchunks = (Kp + Kc - 1) / Kc;
  // columns [k0, k0 + Kc) of the Q rows into shared memory (zero past K)
  auto load_q = [&](int k0) {
    for (int c = 0; c < R; ++c) {
      const float *q = Q + (int64_t)(c < cnt ? (rows ? rows[c] : c) : 0) * ldq;
      for (int k = threadIdx.x; k < Kc; k += blockDim.x)
        qs[c * Kc + k] = c < cnt && k0 + k < K ? q[k0 + k] : 0.0f;
    }
  };
  if (nchunks == 1) {
    load_q(0);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  // NR rows per warp and step: every shared-memory read of Q serves all of them.  The loop count
  // is the same for every warp of the CTA (the chunked path synchronises inside it).
  for (int base = NR * blockIdx.x * warps; base < M; base += NR * gridDim.x * warps) {
    const int m0 = base + NR * (threadIdx.x >> 5);
    const float4 *pr[NR];
#pragma unroll
    for (int t = 0; t < NR; ++t) pr[t] = reinterpret_cast<const float4 *>(P + (int64_t)min(m0 + t, M - 1) * ldp);
    float acc[NR][R];
#pragma unroll
    for (int t = 0; t < NR; ++t)
#pragma unroll
      for (int c = 0; c < R; ++c) acc[t][c] = 0.0f;
    for (int ch = 0; ch < nchunks; ++ch) {
      const int k0 = ch * Kc;
      if (nchunks > 1) {
        __syncthreads();   // the previous chunk is consumed
        load_q(k0);
        __syncthreads();
      }
      const int c4 = min(Kc, Kp - k0) / 4;   // float4 columns of this chunk
#pragma unroll 4
      for (int k4 = lane; k4 < c4; k4 += 32) {
        float4 a[NR];
#pragma unroll
        for (int t = 0; t < NR; ++t) a[t] = m0 < M ? __ldg(pr[t] + k0 / 4 + k4) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int c = 0; c < R; ++c) {
          const float4 q = reinterpret_cast<const float4 *>(qs + c * Kc)[k4];
#pragma unroll
          for (int t = 0; t < NR; ++t) {
            acc[t][c] = fmaf(a[t].x, q.x, acc[t][c]);
            acc[t][c] = fmaf(a[t].y, q.y, acc[t][c]);
            acc[t][c] = fmaf(a[t].z, q.z, acc[t][c]);
            acc[t][c] = fmaf(a[t].w, q.w, acc[t][c]);
          }
        }
      }
    }
    if (m0 >= M) continue;   // uniform over the warp
#pragma unroll
    for (int t = 0; t < NR; ++t)
#pragma unroll
      for (int c = 0; c < R; ++c) acc[t][c] = warp_sum_f(acc[t][c]);
    if (lane < cnt) {
      float *o = out + (int64_t)(rows ? rows[lane] : lane) * ldo;
#pragma unroll
      for (int t = 0; t < NR; ++t) {
        float v = acc[t][0];
#pragma unroll
        for (int c = 1; c < R; ++c)
          if (lane == c) v = acc[t][c];
        if (m0 + t < M) o[m0 + t] = v;
      }
    }
  }
}

// once per kernel and process (thread-safe): the largest shared memory the launcher allows
template <int R, int NR>
cudaError_t gemv_configured() {
  static const cudaError_t e =
      cudaFuncSetAttribute(k_gemv<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemvSmemMax);
  return e;
}

int gemv_width(int r) { return r <= 1 ? 1 : r <= 2 ? 2 : r <= 4 ? 4 : r <= kGemvMaxR ? kGemvMaxR : 0; }

// any K: Q rows that do not fit in shared memory are streamed in chunks
bool gemv_fits(int r, int64_t K) { return gemv_width(r) > 0 && K > 0 && K < INT32_MAX; }

cudaError_t launch_gemv(const float *P, int64_t ldp, int M, int K, const float *Q, int64_t ldq, const int *rows,
                        const int *count, int r, float *out, int64_t ldo, const int *gate, int sms, cudaStream_t st) {
  const int w = gemv_width(r);
  if (w == 0 || K < 1) return cudaErrorInvalidValue;
  const int64_t Kp = (int64_t)(K + 3) / 4 * 4;
  // chunk of the Q rows held in shared memory: all of them when they fit, else the largest
  // multiple of 128 columns that fits (whole float4 steps of every lane)
  int64_t Kc = Kp;
  if ((int64_t)w * Kp * 4 > kGemvSmemMax) Kc = (int64_t)kGemvSmemMax / (4 * w) / 128 * 128;
  const size_t smem = (size_t)w * Kc * sizeof(float);
  // CTAs resident per SM by shared memory (two at least for the streaming), a grid of that many
  // per SM, each CTA loading the Q rows once (per row batch when they are chunked)
  const int per_sm = smem <= 48 * 1024 ? 4 : (smem <= 100 * 1024 ? 2 : 1);
  const int blocks = std::min((M + 15) / 16, per_sm * sms);
  auto go = [&](auto kern, cudaError_t configured) -> cudaError_t {
    if (configured != cudaSuccess) return configured;
    kern<<<blocks, 512, smem, st>>>(P, ldp, M, K, (int)Kc, Q, ldq, rows, count, out, ldo, gate);
    return cudaGetLastError();
  };
  switch (w) {
    case 1: return go(k_gemv<1, 1>, gemv_configured<1, 1>());
    case 2: return go(k_gemv<2, 1>, gemv_configured<2, 1>());
    case 4: return go(k_gemv<4, 2>, gemv_configured<4, 2>());
    default: return go(k_gemv<kGemvMaxR, 2>, gemv_configured<kGemvMaxR, 2>());
  }
}

}  // namespace spca
