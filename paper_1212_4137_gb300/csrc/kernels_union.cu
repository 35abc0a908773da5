// kernels_union.cu -- u = A x (Algorithm 2) when the active starts' supports share few columns.
// After an x-step every x is sparse, and on structured data the starts converge onto a few
// supports, so the union S of the active supports is small.  Then:
//   1. one mark per column of A for every support entry, and an ordered compaction of the
//      marks into S (column -> position, position -> column, K' = |S|), which also decides on
//      the device whether the next sweep takes this path;
//   2. the columns of A in S gathered into the two FP16 planes of the tensor-core format (A's row
//      scales) with the support position contiguous (n x K' per plane, zero-padded to a multiple
//      of 64), from the rows of the FP32 A^T;
//   3. each active x scattered into the same K' positions (two FP16 planes);
// and the tensor-core contraction runs over K' instead of p (work n * K' instead of n * p per
// start, and A is read once instead of once per start).
#include <cuda_fp16.h>

#include <cstdint>

#include "block_util.cuh"
#include "spca_internal.cuh"

namespace spca {

__global__ void __launch_bounds__(256) k_union_mark(const int *__restrict__ sup_idx, int cap, StartState s,
                                                    int *__restrict__ mark) {
  const int c = blockIdx.x;
  if (s.status[c] != ST_ACTIVE) return;
  const int nnz = s.nnz[c];
  const int *gi = sup_idx + (int64_t)c * cap;
  for (int t = threadIdx.x; t < nnz; t += blockDim.x) mark[gi[t]] = 1;
}

// one CTA of 32 warps: warp w owns a contiguous segment of the columns and walks it 32 at a
// time (coalesced), counting marks with ballots; one scan over the 32 warp counts then gives
// every marked column its position in index order
__global__ void __launch_bounds__(1024) k_union_scan(const int *__restrict__ mark, int p, int *__restrict__ colpos,
                                                     int *__restrict__ collist, int kcap, Ctrl *__restrict__ ctrl) {
  __shared__ int woff[32];
  __shared__ int total_s;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int seg = ((p + nw - 1) / nw + 31) / 32 * 32;
  const int lo = min(p, w * seg), hi = min(p, lo + seg);
  int cnt = 0;
  for (int base = lo; base < hi; base += 32) {
    const int j = base + lane;
    cnt += __popc(__ballot_sync(0xffffffffu, j < hi && mark[j] != 0));
  }
  if (lane == 0) woff[w] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int k = 0; k < nw; ++k) { const int t = woff[k]; woff[k] = acc; acc += t; }
    total_s = acc;
  }
  __syncthreads();
  int pos = woff[w];
  const unsigned lt = (1u << lane) - 1u;
  for (int base = lo; base < hi; base += 32) {
    const int j = base + lane;
    const bool on = j < hi && mark[j] != 0;
    const unsigned b = __ballot_sync(0xffffffffu, on);
    if (j < hi) {
      const int q = pos + __popc(b & lt);
      colpos[j] = on ? q : -1;
      if (on && q < kcap) collist[q] = j;
    }
    pos += __popc(b);
  }
  if (threadIdx.x == 0) {
    const int K = total_s;
    ctrl->kunion = K;
    const int use = (ctrl->need_dense == 0 && ctrl->active > 0 && K > 0 && K <= kcap) ? 1 : 0;
    ctrl->use_union = use;
    if (use) ctrl->use_gather = 0;
  }
}

cudaError_t launch_union(const int *sup_idx, int cap, StartState s, int r, int p, int *mark, int *colpos,
                         int *collist, int kcap, Ctrl *c, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(mark, 0, (size_t)p * sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_union_mark<<<r, 256, 0, st>>>(sup_idx, cap, s, mark);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_union_scan<<<1, 1024, 0, st>>>(mark, p, colpos, collist, kcap, c);
  return cudaGetLastError();
}

// AS[t][i * kcap + k] = plane t of a_scale[i] A[i, collist[k]] (= a_scale[i] A^T[collist[k], i])
// for k < K', 0 for K' <= k < kpad: the same operand format as the P planes of A (row scales of
// A), read from the FP32 A^T; 32 x 32 tiles transposed through shared memory (coalesced on both
// sides), visited by a grid-stride loop so that a gated-off launch costs only a few early exits
__global__ void __launch_bounds__(256) k_gather_cols(const float *__restrict__ AT, int64_t ldat,
                                                     const float *__restrict__ a_scale, int n,
                                                     const int *__restrict__ collist, int kcap,
                                                     __half *__restrict__ AS, int64_t as_pstride,
                                                     const Ctrl *__restrict__ ctrl) {
  __shared__ float tile[32][33];
  if (ctrl->use_union == 0) return;
  const int K = ctrl->kunion, kpad = min(kcap, (K + 63) / 64 * 64);
  const int tk = (kpad + 31) / 32, ti = (n + 31) / 32;
  const int ntiles = tk * ti;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int k0 = (t % tk) * 32, i0 = (t / tk) * 32;
    __syncthreads();
    for (int kk = ty; kk < 32; kk += 8) {
      const int k = k0 + kk, i = i0 + tx;
      tile[kk][tx] = (k < K && i < n) ? AT[(int64_t)collist[k] * ldat + i] * a_scale[i] : 0.0f;
    }
    __syncthreads();
    for (int ii = ty; ii < 32; ii += 8) {
      const int i = i0 + ii, k = k0 + tx;
      if (i < n && k < kpad) {
        const float a = tile[tx][ii];
        const __half hi = __float2half_rn(a);
        AS[(int64_t)i * kcap + k] = hi;
        AS[(int64_t)i * kcap + k + as_pstride] = __float2half_rn(a - __half2float(hi));
      }
    }
  }
}

// XS[t][k * kcap + colpos[j]] = plane t of kQScale x_j for the k-th active start (rows zeroed first)
__global__ void __launch_bounds__(256) k_scatter_x(const int *__restrict__ sup_idx, const float *__restrict__ sup_val,
                                                   int cap, StartState s, const int *__restrict__ act,
                                                   const int *__restrict__ colpos, int kcap,
                                                   __half *__restrict__ XS, int64_t xs_pstride,
                                                   const Ctrl *__restrict__ ctrl) {
  if (ctrl->use_union == 0) return;
  const int k = blockIdx.x;
  if (k >= ctrl->active) return;
  const int kpad = min(kcap, (ctrl->kunion + 63) / 64 * 64);
  const int c = act[k];
  __half *row = XS + (int64_t)k * kcap;
  for (int q = threadIdx.x; q < kpad; q += blockDim.x) {
    row[q] = __float2half_rn(0.0f);
    row[q + xs_pstride] = __float2half_rn(0.0f);
  }
  __syncthreads();
  const int nnz = s.nnz[c];
  const int *gi = sup_idx + (int64_t)c * cap;
  const float *gv = sup_val + (int64_t)c * cap;
  for (int t = threadIdx.x; t < nnz; t += blockDim.x) {
    const int pos = colpos[gi[t]];
    if (pos < 0 || pos >= kpad) continue;   // outside the union's first kpad columns (cannot
                                            // happen when use_union is set)
    const float a = gv[t] * kQScale;
    const __half hi = __float2half_rn(a);
    row[pos] = hi;
    row[pos + xs_pstride] = __float2half_rn(a - __half2float(hi));
  }
}

cudaError_t launch_union_operands(const float *AT, int64_t ldat, const float *a_scale, int n, const int *collist,
                                  int kcap, void *AS, int64_t as_pstride, const int *sup_idx,
                                  const float *sup_val, int cap, StartState s, const int *act, int nhost,
                                  const int *colpos, void *XS, int64_t xs_pstride, const Ctrl *c,
                                  cudaStream_t st) {
  k_gather_cols<<<608, 256, 0, st>>>(AT, ldat, a_scale, n, collist, kcap, static_cast<__half *>(AS), as_pstride, c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_scatter_x<<<nhost > 0 ? nhost : 1, 256, 0, st>>>(sup_idx, sup_val, cap, s, act, colpos, kcap,
                                                      static_cast<__half *>(XS), xs_pstride, c);
  return cudaGetLastError();
}

}  // namespace spca
