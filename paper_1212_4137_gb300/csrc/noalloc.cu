// noalloc.cu -- spca_objective_noalloc: the Table 1 objective and explained variance of given
// vectors x, for callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a captured CUDA graph
// being recorded by someone else's framework, under a memory pool or allocator that owns the
// whole device, or in a real-time loop where an allocation's implicit synchronisation and
// latency are not acceptable.  Such a caller already holds A, the x's and the result arrays in
// device memory; this entry point adds nothing to the device heap.
//
// The computation is the one spca_solve reports per start (u = A x with FP64 products and sums,
// then the objective of the formulation and ||Ax||_2^2 or ||Ax||_1), done by a variant of the
// finalisation kernels whose per-(start, row chunk) partial sums live in a file-scope
// __device__ array instead of handle memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "block_util.cuh"
#include "spca_internal.cuh"

namespace spca {
namespace {

constexpr int NT = 256;                 // rows of A per CTA (a chunk), and threads per CTA
constexpr int NW = NT / 32;             // warps per CTA; warp w takes rows w, w + NW, ... of the chunk
constexpr int RPW = NT / NW;            // rows per warp (32)
constexpr int XCHUNK = 1024;            // nonzeros of x staged in shared memory at a time

// the scratch: (r * ceil(n / 256)) pairs of doubles, at most SPCA_NOALLOC_MAX_PARTIALS pairs.
// Every GPU that loads the library holds these 4 MiB until the process exits.
__device__ __align__(256) double g_partials[2 * SPCA_NOALLOC_MAX_PARTIALS];

// grid (nchunks, r): u_i = sum_j x_j A[i, j] over the nonzeros of x, products and sums in FP64,
// for the 256 rows of chunk b; this CTA's sums of |u_i| and u_i^2 go to
// partials[(c * nchunks + b) * 2].  A warp owns 32 rows; for each row its lanes walk the staged
// nonzeros of x together (lane t reads column sj[t], and the staged columns ascend, so a warp's
// loads of one row are contiguous when x is dense), each lane keeping one FP64 sum per row that
// the warp adds up in a fixed order at the end.
__global__ void __launch_bounds__(NT) k_obj_partial(const float *__restrict__ A, int64_t lda, int n, int p,
                                                    const float *__restrict__ X, int64_t ldx,
                                                    double *__restrict__ partials) {
  __shared__ int sj[XCHUNK];
  __shared__ float sx[XCHUNK];
  __shared__ int red_i[32];
  __shared__ double red[32];
  const int c = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int row0 = blockIdx.x * NT;
  const float *x = X + (int64_t)c * ldx;
  double acc[RPW];
#pragma unroll
  for (int k = 0; k < RPW; ++k) acc[k] = 0.0;
  // walk x in chunks of NT entries; stage its nonzeros (in index order) and use them
  int staged = 0;
  for (int base = 0; base < p; base += NT) {
    const int j = base + threadIdx.x;
    const float xj = j < p ? x[j] : 0.0f;
    int tot;
    const int pos = staged + block_excl_scan_flag(xj != 0.0f, red_i, &tot);
    if (xj != 0.0f) {
      sj[pos] = j;
      sx[pos] = xj;
    }
    staged += tot;
    // flush when the staging buffer could overflow on the next chunk, or at the end
    if (staged > XCHUNK - NT || base + NT >= p) {
      __syncthreads();
#pragma unroll
      for (int k = 0; k < RPW; ++k) {
        const int i = row0 + w + k * NW;
        if (i < n) {
          const float *arow = A + (int64_t)i * lda;
          for (int t = lane; t < staged; t += 32) acc[k] = fma((double)sx[t], (double)arow[sj[t]], acc[k]);
        }
      }
      __syncthreads();
      staged = 0;
    }
  }
  // u_i for the warp's rows (lane sums added in a fixed order), then |u_i| and u_i^2
  double l1 = 0.0, l2 = 0.0;
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const double u = warp_sum_d(acc[k]);
    if (row0 + w + k * NW < n) {
      l1 += fabs(u);
      l2 += u * u;
    }
  }
  // every lane holds the warp's sums: lane 0 of each warp contributes them
  l1 = block_sum_d(lane == 0 ? l1 : 0.0, red);
  l2 = block_sum_d(lane == 0 ? l2 : 0.0, red);
  if (threadIdx.x == 0) {
    double *o = partials + ((int64_t)c * gridDim.x + blockIdx.x) * 2;
    o[0] = l1;
    o[1] = l2;
  }
}

// one thread per start: the partials in chunk order, ||x||_0, ||x||_1, then the objective
__global__ void __launch_bounds__(NT) k_obj_reduce(int form, double gamma, const double *__restrict__ partials,
                                                   int nchunks, const float *__restrict__ X, int64_t ldx, int p,
                                                   int r, double *__restrict__ f, double *__restrict__ ev) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= r) return;
  double l1 = 0.0, l2sq = 0.0, x0 = 0.0, x1 = 0.0;
  for (int b = 0; b < nchunks; ++b) {
    l1 += partials[((int64_t)c * nchunks + b) * 2 + 0];
    l2sq += partials[((int64_t)c * nchunks + b) * 2 + 1];
  }
  const float *x = X + (int64_t)c * ldx;
  for (int j = 0; j < p; ++j) {
    x0 += (x[j] != 0.0f);
    x1 += fabs((double)x[j]);
  }
  const double l2 = sqrt(l2sq);
  double val;
  switch (form) {
    case 1: case 3: val = l2; break;
    case 2: case 4: val = l1; break;
    case 5: val = l2sq - gamma * x0; break;
    case 6: val = l1 * l1 - gamma * x0; break;
    case 7: val = l2 - gamma * x1; break;
    default: val = l1 - gamma * x1; break;
  }
  f[c] = val;
  ev[c] = is_l1_var(form) ? l1 : l2sq;
}

// set-up once per device (with that device current): the device address of the scratch
std::mutex g_mu;
double *g_addr[64] = {nullptr};

cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_partials);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double *>(ptr);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace spca

using namespace spca;

extern "C" int spca_objective_noalloc(int form, double gamma, const float *A, int64_t n, int64_t p, int64_t lda,
                                      const float *X, int64_t ldx, int r, double *f, double *ev,
                                      void *cuda_stream) {
  if (form < 1 || form > 8 || !A || !X || !f || !ev) return SPCA_E_INVALID;
  if (n < 1 || p < 1 || r < 1 || lda < p || ldx < p || n > INT32_MAX || p > INT32_MAX) return SPCA_E_INVALID;
  if (!std::isfinite(gamma) || gamma < 0.0) return SPCA_E_INVALID;
  if (r > spca::kMaxStarts) return SPCA_E_UNSUPPORTED;   // the starts ride on the grid's y dimension
  const int64_t nchunks = (n + NT - 1) / NT;
  if ((int64_t)r * nchunks > (int64_t)SPCA_NOALLOC_MAX_PARTIALS) return SPCA_E_INVALID;   // beyond the scratch
  double *partials = nullptr;
  if (scratch_for_current_device(&partials) != cudaSuccess) return SPCA_E_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // every partial the reduction reads is written by this call's first kernel (no zeroing needed)
  k_obj_partial<<<dim3((unsigned)nchunks, (unsigned)r), NT, 0, st>>>(A, lda, (int)n, (int)p, X, ldx, partials);
  if (cudaGetLastError() != cudaSuccess) return SPCA_E_CUDA;
  k_obj_reduce<<<(r + NT - 1) / NT, NT, 0, st>>>(form, gamma, partials, (int)nchunks, X, ldx, (int)p, r, f, ev);
  if (cudaGetLastError() != cudaSuccess) return SPCA_E_CUDA;
  return SPCA_OK;
}
