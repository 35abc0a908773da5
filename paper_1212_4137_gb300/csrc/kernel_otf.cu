// kernel_otf.cu -- on-the-fly replacement of converged starts (Section 4.3): a solve of l starts
// runs them through r slots; a slot whose start has stopped (converged, degenerate or out of
// sweeps) archives that start's result and takes the next start, so that the contractions keep
// working on r starts until fewer than r are left.
//   k_otf_retire   after the x-step: archives the scalars of every stopped slot (F, sweeps, status,
//                  gamma, nnz), lists the stopped slots in slot order, and gives the next starts
//                  to the first of them (the others stay idle);
//   k_otf_archive  copies the stopped slots' x to the archive (the new starts' x overwrites them
//                  next, in the start initialisation over the new-slot list);
//   k_otf_obj / k_otf_reduce
//                  after the sweeps: the Table 1 objective and explained variance of every
//                  archived start in compensated FP32-pair accumulation (the finalise's), and its
//                  u = A x, from which the best start's y follows.
#include <cstdint>

#include "block_util.cuh"
#include "spca_internal.cuh"

namespace spca {

__global__ void __launch_bounds__(1024) k_otf_retire(int r, int l, StartState s, int *__restrict__ slot_start,
                                                     int *__restrict__ next_start, OtfArchive arc,
                                                     int *__restrict__ retire_slot, int *__restrict__ retire_start,
                                                     int *__restrict__ new_slot, Ctrl *__restrict__ ctrl) {
  __shared__ int red[32];
  const int next0 = *next_start;
  int base = 0;
  for (int c0 = 0; c0 < r; c0 += blockDim.x) {
    const int c = c0 + threadIdx.x;
    const bool ret = c < r && slot_start[c] >= 0 && s.status[c] != ST_ACTIVE;
    int tot;
    const int pos = base + block_excl_scan_flag(ret, red, &tot);
    if (ret) {
      const int st = slot_start[c];
      arc.F[st] = s.F[c];
      arc.iters[st] = s.iters[c];
      arc.status[st] = s.status[c];
      arc.gamma[st] = s.gamma[c];
      arc.nnz[st] = s.nnz[c];
      retire_slot[pos] = c;
      retire_start[pos] = st;
      const int id = next0 + pos;
      if (id < l) {
        new_slot[pos] = c;
        slot_start[c] = id;
      } else {
        slot_start[c] = -1;   // no start left: the slot stays idle
      }
    }
    base += tot;
  }
  if (threadIdx.x == 0) {
    const int n_new = max(0, min(base, l - next0));
    ctrl->n_retire = base;
    ctrl->n_new = n_new;
    *next_start = next0 + n_new;
  }
}

__global__ void __launch_bounds__(256) k_otf_archive(const float *__restrict__ X, int64_t ldx, int p,
                                                     const int *__restrict__ retire_slot,
                                                     const int *__restrict__ retire_start,
                                                     const Ctrl *__restrict__ ctrl, float *__restrict__ arc_x) {
  const int k = blockIdx.x;
  if (k >= ctrl->n_retire) return;
  const float *src = X + (int64_t)retire_slot[k] * ldx;
  float *dst = arc_x + (int64_t)retire_start[k] * ldx;
  for (int j = threadIdx.x; j < p; j += blockDim.x) dst[j] = src[j];
}

cudaError_t launch_otf_retire(int r, int l, StartState s, int *slot_start, int *next_start, OtfArchive arc,
                              int *retire_slot, int *retire_start, int *new_slot, Ctrl *ctrl, const float *X,
                              int64_t ldx, int p, cudaStream_t st) {
  k_otf_retire<<<1, 1024, 0, st>>>(r, l, s, slot_start, next_start, arc, retire_slot, retire_start, new_slot, ctrl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_otf_archive<<<r, 256, 0, st>>>(X, ldx, p, retire_slot, retire_start, ctrl, arc.x);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- objectives of the archive
namespace {
constexpr int OT = 256;
constexpr int OCHUNK = 1024;   // nonzeros of x staged per round
}

// grid (ceil(n / OT), l): u_i = sum_j x_j A[i, j] over the nonzeros of archived x (ascending j),
// compensated FP32 pairs; u to arc.U; per-CTA FP64 sums of |u_i| and u_i^2 to partials
__global__ void __launch_bounds__(OT) k_otf_obj(const float *__restrict__ AT, int64_t ldat, int n, int p,
                                                OtfArchive arc, int64_t ldx, int64_t ldu,
                                                double *__restrict__ partials) {
  __shared__ int sj[OCHUNK];
  __shared__ float sx[OCHUNK];
  __shared__ int red_i[32];
  __shared__ double red[32];
  const int c = blockIdx.y;
  const int i = blockIdx.x * OT + threadIdx.x;
  const float *x = arc.x + (int64_t)c * ldx;
  F32Pair acc;
  int staged = 0;
  for (int base = 0; base < p; base += OT) {
    const int j = base + threadIdx.x;
    const float xj = j < p ? x[j] : 0.0f;
    int tot;
    const int pos = staged + block_excl_scan_flag(xj != 0.0f, red_i, &tot);
    if (xj != 0.0f) {
      sj[pos] = j;
      sx[pos] = xj;
    }
    staged += tot;
    if (staged > OCHUNK - OT || base + OT >= p) {
      __syncthreads();
      if (i < n)
        for (int t = 0; t < staged; ++t) f32pair_fma(acc, sx[t], AT[(int64_t)sj[t] * ldat + i]);
      __syncthreads();
      staged = 0;
    }
  }
  const double u = f32pair_value(acc);
  if (i < n) arc.U[(int64_t)c * ldu + i] = (float)u;
  const double l1 = block_sum_d(i < n ? fabs(u) : 0.0, red);
  const double l2 = block_sum_d(i < n ? u * u : 0.0, red);
  if (threadIdx.x == 0) {
    double *o = partials + ((int64_t)c * gridDim.x + blockIdx.x) * 2;
    o[0] = l1;
    o[1] = l2;
  }
}

// block per start: the partials in order, ||x||_0 and ||x||_1, then f (Table 1) and the
// explained variance (the archive's starts, or a solve's starts with a sparse A)
__global__ void __launch_bounds__(OT) k_otf_reduce(int form, const double *__restrict__ partials, int nchunks,
                                                   int p, OtfArchive arc, int64_t ldx) {
  __shared__ double red[32];
  __shared__ int red_i[32];
  const int c = blockIdx.x;
  const float *x = arc.x + (int64_t)c * ldx;
  double a1 = 0.0;
  int nz = 0;
  for (int j = threadIdx.x; j < p; j += OT) {
    a1 += fabs((double)x[j]);
    nz += x[j] != 0.0f;
  }
  const double x1 = block_sum_d(a1, red);
  const int x0 = block_sum_i(nz, red_i);
  if (threadIdx.x != 0) return;
  double l1 = 0.0, l2sq = 0.0;
  for (int b = 0; b < nchunks; ++b) {
    l1 += partials[((int64_t)c * nchunks + b) * 2 + 0];
    l2sq += partials[((int64_t)c * nchunks + b) * 2 + 1];
  }
  const double l2 = sqrt(l2sq), g = arc.gamma[c];
  double f;
  switch (form) {
    case 1: case 3: f = l2; break;
    case 2: case 4: f = l1; break;
    case 5: f = l2sq - g * (double)x0; break;
    case 6: f = l1 * l1 - g * (double)x0; break;
    case 7: f = l2 - g * x1; break;
    default: f = l1 - g * x1; break;
  }
  arc.f[c] = f;
  arc.ev[c] = is_l1_var(form) ? l1 : l2sq;
}

cudaError_t launch_otf_objectives(int form, const float *AT, int64_t ldat, int n, int p, OtfArchive arc, int l,
                                  int64_t ldx, int64_t ldu, double *partials, cudaStream_t st) {
  const int nchunks = (n + OT - 1) / OT;
  k_otf_obj<<<dim3((unsigned)nchunks, (unsigned)l), OT, 0, st>>>(AT, ldat, n, p, arc, ldx, ldu, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_objective_reduce(form, partials, nchunks, p, arc, l, ldx, st);
}

cudaError_t launch_objective_reduce(int form, const double *partials, int nchunks, int p, OtfArchive arc, int count,
                                    int64_t ldx, cudaStream_t st) {
  k_otf_reduce<<<count, OT, 0, st>>>(form, partials, nchunks, p, arc, ldx);
  return cudaGetLastError();
}

}  // namespace spca
