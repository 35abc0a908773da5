// kernels_sparse.cu -- the products of an AM sweep (Algorithm 2) for a sparse A held in compressed
// sparse rows, the layout of the text corpora of Section 5 (document x word counts).  The handle
// keeps A by rows (CSR of A, n rows) and by columns (CSR of A^T, p rows); both are canonical
// (indices ascending within a row, no repeats).
//
//   k_pack_t        B^T of the listed rows of X or Y, packed start-fastest: Bt[j * ldb + k] =
//                   src[list[k]][j], so that one stored entry of A meets 8 starts in one 32-byte
//                   sector of Bt;
//   k_spmm          out[list[k]][row] = sum over the row's entries a_{row,j} Bt[j][k] (u = A x with
//                   A by rows and a dense x; v = A^T y with A by columns), up to 32 starts.  Work
//                   items of at most kSpItemNnz entries (a run of short rows, or a segment of a
//                   long row) are taken by warps; a warp walks an item once, each lane keeping 8
//                   FP32 sums per group of 8 starts over a strided subset of the entries, then the
//                   warp reduces each group (reduce-scatter: lane L ends with start L / 4);
//   k_spmm_wide     the same for many starts (more than 32): the starts are cut into slabs of 64,
//                   slab-major, so that the slab of Bt the warps gather from (64 starts x the
//                   operand's length) stays in L2; a warp takes an item of a slab, its lanes own 2
//                   starts each and walk the item's entries in order (each entry's index and value
//                   broadcast from the lane that loaded it), reading one 256-byte row segment of Bt
//                   per entry;
//   k_pack_t_h, k_spmm_h, k_spmm_wide_h
//                   the same for y = +-1 (L1 variance), which FP16 holds exactly: 16 starts per
//                   32-byte sector (slabs of 128 starts), products and sums in FP32;
//   k_spmm_fix      a long row's segments' sums added in segment order;
//   k_spmv_support  u = A x over the support of a sparse x: the support's columns (A^T's rows)
//                   scattered into a shared-memory chunk of u, one column at a time in support
//                   order, the FMA chain of each u_i in that order;
//   k_fin_support   the finalise's u = A x in compensated FP32 pairs over a small support (the
//                   column scatter into 256-row chunks), |u| and u^2 summed in pair arithmetic;
//   k_fin_csr       the same by rows for the other starts, 8 starts per pass over a row;
//   k_lowrank_*     projection deflation of a sparse A kept as a low-rank update: after k
//                   components, A_k = A (I - z_1 z_1^T) ... (I - z_k z_k^T) = A - W Z^T with z_i
//                   unit and w_i = A_{i-1} z_i, so u = A x - W (Z^T x) and v = A^T y - Z (W^T y)
//                   (the finalise subtracts W (Z^T x) in pair arithmetic before its sums).
// Every sum runs in a fixed order: a start's result does not depend on the schedule or on the
// other starts.
#include <cuda_fp16.h>

#include <cstdint>

#include "block_util.cuh"
#include "spca_internal.cuh"

namespace spca {

namespace {
constexpr int SPT = 256;            // threads per CTA of the SpMM
constexpr int SCH = 4096;           // rows of u per CTA of the support scatter
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void fma8v(float (&acc)[8], float a, const float (&x)[8]) {
#pragma unroll
  for (int t = 0; t < 8; ++t) acc[t] = fmaf(a, x[t], acc[t]);
}

// one 32-byte load (sm_100+: 256-bit vector loads; p 32-byte aligned) through the non-coherent
// path: the 8 starts of a packed row segment in one L1 request instead of two
__device__ __forceinline__ void ldg8(const float *p, float (&v)[8]) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}

// the same load as raw 32-bit words (16 FP16 values)
__device__ __forceinline__ void ldg8u(const void *p, uint32_t (&v)[8]) {
  asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
      : "l"(p));
}
__device__ __forceinline__ float2 half2_bits(uint32_t u) {
  __half2 h;
  memcpy(&h, &u, sizeof h);
  return __half22float2(h);
}

// Sum over the warp of a[q] for q = (lane >> 1) & 15, in 16 shuffles (the levels 16, 8, 4 and 2
// halve the values a lane keeps, as in reduce8 below)
__device__ __forceinline__ float reduce16(const float (&a)[16], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float t8[8], t4[4], t2[2];
#pragma unroll
  for (int q = 0; q < 8; ++q) t8[q] = (b4 ? a[q + 8] : a[q]) + __shfl_xor_sync(FULL, b4 ? a[q] : a[q + 8], 16);
#pragma unroll
  for (int q = 0; q < 4; ++q) t4[q] = (b3 ? t8[q + 4] : t8[q]) + __shfl_xor_sync(FULL, b3 ? t8[q] : t8[q + 4], 8);
#pragma unroll
  for (int q = 0; q < 2; ++q) t2[q] = (b2 ? t4[q + 2] : t4[q]) + __shfl_xor_sync(FULL, b2 ? t4[q] : t4[q + 2], 4);
  float w = (b1 ? t2[1] : t2[0]) + __shfl_xor_sync(FULL, b1 ? t2[0] : t2[1], 2);
  w += __shfl_xor_sync(FULL, w, 1);
  return w;
}

// Sum over the warp of a[q] for q = (lane >> 2) & 7, in 9 shuffles: at each of the levels 16, 8
// and 4 a lane keeps half of its values, adds its partner's copy of them and hands over the
// other half; levels 2 and 1 finish the sum.  Both lanes of a pair form the same sum.
__device__ __forceinline__ float reduce8(const float (&a)[8], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float t[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float send = b4 ? a[q] : a[q + 4];
    const float keep = b4 ? a[q + 4] : a[q];
    t[q] = keep + __shfl_xor_sync(FULL, send, 16);
  }
  float u[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float send = b3 ? t[q] : t[q + 2];
    const float keep = b3 ? t[q + 2] : t[q];
    u[q] = keep + __shfl_xor_sync(FULL, send, 8);
  }
  float w = (b2 ? u[1] : u[0]) + __shfl_xor_sync(FULL, b2 ? u[0] : u[1], 4);
  w += __shfl_xor_sync(FULL, w, 2);
  w += __shfl_xor_sync(FULL, w, 1);
  return w;
}

// first k in [b, e) with col[k] >= v (col ascending on [b, e))
__device__ __forceinline__ int64_t lower_bound_col(const int *__restrict__ col, int64_t b, int64_t e, int v) {
  while (b < e) {
    const int64_t m = b + ((e - b) >> 1);
    if (col[m] < v) b = m + 1;
    else e = m;
  }
  return b;
}
}  // namespace

// grid (ceil(len / 32), ceil(rmax / 32)), block (32, 8): a 32 x 32 tile through shared memory
__global__ void k_pack_t(const float *__restrict__ src, int64_t ld, int len, const int *__restrict__ list,
                         const int *__restrict__ count, int rmax, const int *__restrict__ gate,
                         float *__restrict__ Bt, int ldb) {
  if (gate && *gate == 0) return;
  const int cnt = count ? *count : rmax;
  const int k0 = blockIdx.y * 32;
  const int kpad = (cnt + kSpGroup - 1) / kSpGroup * kSpGroup;
  if (k0 >= kpad) return;
  __shared__ float tile[32][33];
  const int j0 = blockIdx.x * 32;
  for (int q = threadIdx.y; q < 32; q += 8) {
    const int k = k0 + q, j = j0 + threadIdx.x;
    float v = 0.0f;
    if (k < cnt && j < len) v = src[(int64_t)(list ? list[k] : k) * ld + j];
    tile[q][threadIdx.x] = v;
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += 8) {
    const int j = j0 + q, k = k0 + threadIdx.x;
    if (j < len && k < kpad) Bt[(int64_t)j * ldb + k] = tile[threadIdx.x][q];
  }
}

cudaError_t launch_pack_t(const float *src, int64_t ld, int len, const int *list, const int *count,
                          const int *gate, int rmax, float *Bt, int ldb, cudaStream_t st) {
  const dim3 grid((unsigned)((len + 31) / 32), (unsigned)((rmax + 31) / 32));
  k_pack_t<<<grid, dim3(32, 8), 0, st>>>(src, ld, len, list, count, rmax, gate, Bt, ldb);
  return cudaGetLastError();
}

// NG groups of 8 starts per pass over an item's entries (the host takes NG = ceil(rmax / 8) <= 4):
// each entry's index and value are loaded once for all of them
template <int NG>
__global__ void __launch_bounds__(SPT) k_spmm(SpMat M, const SpItem *__restrict__ items, int nitems,
                                              const float *__restrict__ Bt, int ldb, const int *__restrict__ count,
                                              const int *__restrict__ gate, const int *__restrict__ list,
                                              float *__restrict__ out, int64_t ldo, float *__restrict__ part) {
  if (gate && *gate == 0) return;
  const int cnt = *count;
  if (cnt <= 0) return;
  const int ng = min(NG, (cnt + kSpGroup - 1) / kSpGroup);
  const int lane = threadIdx.x & 31, q = lane >> 2;
  const int nw = gridDim.x * (SPT / 32);
  for (int it = blockIdx.x * (SPT / 32) + (threadIdx.x >> 5); it < nitems; it += nw) {
    const int4 head = __ldg(reinterpret_cast<const int4 *>(items + it));   // row0, row1, seg
    const int seg = head.z;
    for (int row = head.x; row < head.y; ++row) {
      const int64_t b = seg >= 0 ? items[it].nz0 : M.ptr[row];
      const int64_t e = seg >= 0 ? items[it].nz1 : M.ptr[row + 1];
      float acc[NG][8];
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[g][t] = 0.0f;
      int64_t k = b + lane;
      // two entries per lane in flight; each lane's sums still run in entry order
      for (; k + 32 < e; k += 64) {
        const int j0 = __ldg(M.col + k), j1 = __ldg(M.col + k + 32);
        const float a0 = __ldg(M.val + k), a1 = __ldg(M.val + k + 32);
        const float *p0 = Bt + (int64_t)j0 * ldb, *p1 = Bt + (int64_t)j1 * ldb;
        float x0[NG][8], x1[NG][8];
#pragma unroll
        for (int g = 0; g < NG; ++g)
          if (g < ng) {
            ldg8(p0 + 8 * g, x0[g]);
            ldg8(p1 + 8 * g, x1[g]);
          }
#pragma unroll
        for (int g = 0; g < NG; ++g)
          if (g < ng) {
            fma8v(acc[g], a0, x0[g]);
            fma8v(acc[g], a1, x1[g]);
          }
      }
      if (k < e) {
        const int j0 = __ldg(M.col + k);
        const float a0 = __ldg(M.val + k);
        const float *p0 = Bt + (int64_t)j0 * ldb;
#pragma unroll
        for (int g = 0; g < NG; ++g)
          if (g < ng) {
            float x0[8];
            ldg8(p0 + 8 * g, x0);
            fma8v(acc[g], a0, x0);
          }
      }
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        if (g >= ng) break;
        const float v = reduce8(acc[g], lane);
        const int kk = g * kSpGroup + q;
        if ((lane & 3) == 0 && kk < cnt) {
          if (seg >= 0) part[(int64_t)seg * ldb + kk] = v;
          else out[(int64_t)(list ? list[kk] : kk) * ldo + row] = v;
        }
      }
    }
  }
}

constexpr int kWideSlab = 64;   // starts per slab of k_spmm_wide (2 per lane)

__global__ void __launch_bounds__(SPT, 3) k_spmm_wide(SpMat M, const SpItem *__restrict__ items, int nitems,
                                                   const float *__restrict__ Bt, int ldb,
                                                   const int *__restrict__ count, const int *__restrict__ gate,
                                                   const int *__restrict__ list, float *__restrict__ out,
                                                   int64_t ldo, float *__restrict__ part) {
  if (gate && *gate == 0) return;
  const int cnt = *count;
  if (cnt <= 0) return;
  const int lane = threadIdx.x & 31;
  const int nslab = (cnt + kWideSlab - 1) / kWideSlab;
  const int64_t units = (int64_t)nslab * nitems;
  const int64_t nw = (int64_t)gridDim.x * (SPT / 32);
  for (int64_t w = (int64_t)blockIdx.x * (SPT / 32) + (threadIdx.x >> 5); w < units; w += nw) {
    const int slab = (int)(w / nitems), it = (int)(w - (int64_t)slab * nitems);
    const int k = slab * kWideSlab + 2 * lane;      // this lane's two starts: k, k + 1
    const bool on = k < cnt;                        // k + 1 < ldb whenever k < cnt (both even-aligned)
    const float *B = Bt + k;
    const int4 head = __ldg(reinterpret_cast<const int4 *>(items + it));   // row0, row1, seg
    const int seg = head.z;
    for (int row = head.x; row < head.y; ++row) {
      const int64_t b = seg >= 0 ? items[it].nz0 : M.ptr[row];
      const int64_t e = seg >= 0 ? items[it].nz1 : M.ptr[row + 1];
      float2 acc = make_float2(0.0f, 0.0f);
      for (int64_t base = b; base < e; base += 32) {
        const int m = (int)min((int64_t)32, e - base);
        const int jl = lane < m ? __ldg(M.col + base + lane) : 0;
        const float al = lane < m ? __ldg(M.val + base + lane) : 0.0f;
        int q = 0;
        // eight entries' loads in flight, summed in entry order
        for (; q + 8 <= m; q += 8) {
          float2 y[8];
          float a[8];
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            const int j = __shfl_sync(FULL, jl, q + g);
            a[g] = __shfl_sync(FULL, al, q + g);
            y[g] = on ? __ldg(reinterpret_cast<const float2 *>(B + (int64_t)j * ldb)) : make_float2(0.0f, 0.0f);
          }
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            acc.x = fmaf(a[g], y[g].x, acc.x);
            acc.y = fmaf(a[g], y[g].y, acc.y);
          }
        }
        for (; q < m; ++q) {
          const int j = __shfl_sync(FULL, jl, q);
          const float a = __shfl_sync(FULL, al, q);
          const float2 y = on ? __ldg(reinterpret_cast<const float2 *>(B + (int64_t)j * ldb)) : make_float2(0.0f, 0.0f);
          acc.x = fmaf(a, y.x, acc.x);
          acc.y = fmaf(a, y.y, acc.y);
        }
      }
      if (on) {
        if (seg >= 0) {
          part[(int64_t)seg * ldb + k] = acc.x;
          if (k + 1 < cnt) part[(int64_t)seg * ldb + k + 1] = acc.y;
        } else {
          out[(int64_t)(list ? list[k] : k) * ldo + row] = acc.x;
          if (k + 1 < cnt) out[(int64_t)(list ? list[k + 1] : k + 1) * ldo + row] = acc.y;
        }
      }
    }
  }
}

// block per long row: its segments' sums in segment order
__global__ void __launch_bounds__(256) k_spmm_fix(const SpLong *__restrict__ longs, const float *__restrict__ part,
                                                  int ldb, const int *__restrict__ count,
                                                  const int *__restrict__ gate, const int *__restrict__ list,
                                                  float *__restrict__ out, int64_t ldo) {
  if (gate && *gate == 0) return;
  const int cnt = *count;
  const SpLong L = longs[blockIdx.x];
  for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
    float s = 0.0f;
    for (int g = 0; g < L.nseg; ++g) s += part[(int64_t)(L.seg0 + g) * ldb + k];
    out[(int64_t)(list ? list[k] : k) * ldo + L.row] = s;
  }
}

cudaError_t launch_spmm(SpMat M, const SpPlan &P, const float *Bt, int ldb, const int *count, const int *gate,
                        const int *list, int rmax, float *out, int64_t ldo, float *part, int sms, cudaStream_t st) {
  if (P.nitems > 0) {
    // up to 32 starts: lanes over entries (8 starts per 32-byte sector); more: slabs of 64 starts,
    // lanes over starts
    const bool wide = rmax > 32;
    const int64_t units = (int64_t)P.nitems * (wide ? (rmax + kWideSlab - 1) / kWideSlab : 1);
    const int64_t want = (units + SPT / 32 - 1) / (SPT / 32);
    const int blocks = (int)(want < sms * 8 ? want : sms * 8);
    if (wide)
      k_spmm_wide<<<blocks, SPT, 0, st>>>(M, P.items, P.nitems, Bt, ldb, count, gate, list, out, ldo, part);
    else if (rmax <= 8)
      k_spmm<1><<<blocks, SPT, 0, st>>>(M, P.items, P.nitems, Bt, ldb, count, gate, list, out, ldo, part);
    else if (rmax <= 16)
      k_spmm<2><<<blocks, SPT, 0, st>>>(M, P.items, P.nitems, Bt, ldb, count, gate, list, out, ldo, part);
    else if (rmax <= 24)
      k_spmm<3><<<blocks, SPT, 0, st>>>(M, P.items, P.nitems, Bt, ldb, count, gate, list, out, ldo, part);
    else
      k_spmm<4><<<blocks, SPT, 0, st>>>(M, P.items, P.nitems, Bt, ldb, count, gate, list, out, ldo, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (P.nlong > 0) {
    k_spmm_fix<<<P.nlong, 256, 0, st>>>(P.longs, part, ldb, count, gate, list, out, ldo);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------- y = +-1 in FP16
// Bt16[j * ldb + k] = fp16(src[list[k]][j]) (exact for +-1), zero up to the next multiple of 16
__global__ void k_pack_t_h(const float *__restrict__ src, int64_t ld, int len, const int *__restrict__ list,
                           const int *__restrict__ count, __half *__restrict__ Bt, int ldb) {
  const int cnt = *count;
  const int k0 = blockIdx.y * 32;
  const int kpad = (cnt + 15) / 16 * 16;
  if (k0 >= kpad) return;
  __shared__ float tile[32][33];
  const int j0 = blockIdx.x * 32;
  for (int q = threadIdx.y; q < 32; q += 8) {
    const int k = k0 + q, j = j0 + threadIdx.x;
    float v = 0.0f;
    if (k < cnt && j < len) v = src[(int64_t)(list ? list[k] : k) * ld + j];
    tile[q][threadIdx.x] = v;
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += 8) {
    const int j = j0 + q, k = k0 + threadIdx.x;
    if (j < len && k < kpad) Bt[(int64_t)j * ldb + k] = __float2half_rn(tile[threadIdx.x][q]);
  }
}

// up to 32 starts: NG groups of 16 per pass over the entries, one 256-bit load per group
template <int NG>
__global__ void __launch_bounds__(SPT) k_spmm_h(SpMat M, const SpItem *__restrict__ items, int nitems,
                                                const __half *__restrict__ Bt, int ldb,
                                                const int *__restrict__ count, const int *__restrict__ list,
                                                float *__restrict__ out, int64_t ldo, float *__restrict__ part,
                                                int ldp) {
  const int cnt = *count;
  if (cnt <= 0) return;
  const int ng = min(NG, (cnt + 15) / 16);
  const int lane = threadIdx.x & 31, q = lane >> 1;
  const int nw = gridDim.x * (SPT / 32);
  for (int it = blockIdx.x * (SPT / 32) + (threadIdx.x >> 5); it < nitems; it += nw) {
    const int4 head = __ldg(reinterpret_cast<const int4 *>(items + it));
    const int seg = head.z;
    for (int row = head.x; row < head.y; ++row) {
      const int64_t b = seg >= 0 ? items[it].nz0 : M.ptr[row];
      const int64_t e = seg >= 0 ? items[it].nz1 : M.ptr[row + 1];
      float acc[NG][16];
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int t = 0; t < 16; ++t) acc[g][t] = 0.0f;
      auto fma16 = [&](float (&ac)[16], float a, const uint32_t (&w)[8]) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const float2 y2 = half2_bits(w[t]);
          ac[2 * t] = fmaf(a, y2.x, ac[2 * t]);
          ac[2 * t + 1] = fmaf(a, y2.y, ac[2 * t + 1]);
        }
      };
      int64_t k = b + lane;
      // two entries per lane in flight; each lane's sums still run in entry order
      for (; k + 32 < e; k += 64) {
        const int j0 = __ldg(M.col + k), j1 = __ldg(M.col + k + 32);
        const float a0 = __ldg(M.val + k), a1 = __ldg(M.val + k + 32);
        const __half *p0 = Bt + (int64_t)j0 * ldb, *p1 = Bt + (int64_t)j1 * ldb;
        uint32_t w0[NG][8], w1[NG][8];
#pragma unroll
        for (int g = 0; g < NG; ++g)
          if (g < ng) {
            ldg8u(p0 + 16 * g, w0[g]);
            ldg8u(p1 + 16 * g, w1[g]);
          }
#pragma unroll
        for (int g = 0; g < NG; ++g)
          if (g < ng) {
            fma16(acc[g], a0, w0[g]);
            fma16(acc[g], a1, w1[g]);
          }
      }
      if (k < e) {
        const int j0 = __ldg(M.col + k);
        const float a0 = __ldg(M.val + k);
        const __half *p0 = Bt + (int64_t)j0 * ldb;
#pragma unroll
        for (int g = 0; g < NG; ++g)
          if (g < ng) {
            uint32_t w0[8];
            ldg8u(p0 + 16 * g, w0);
            fma16(acc[g], a0, w0);
          }
      }
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        if (g >= ng) break;
        const float v = reduce16(acc[g], lane);
        const int kk = g * 16 + q;
        if ((lane & 1) == 0 && kk < cnt) {
          if (seg >= 0) part[(int64_t)seg * ldp + kk] = v;
          else out[(int64_t)(list ? list[kk] : kk) * ldo + row] = v;
        }
      }
    }
  }
}

// more than 32 starts: slabs of 128 starts, each lane 4 (one 8-byte load per entry)
constexpr int kWideSlabH = 128;
__global__ void __launch_bounds__(SPT, 3) k_spmm_wide_h(SpMat M, const SpItem *__restrict__ items, int nitems,
                                                        const __half *__restrict__ Bt, int ldb,
                                                        const int *__restrict__ count, const int *__restrict__ list,
                                                        float *__restrict__ out, int64_t ldo,
                                                        float *__restrict__ part, int ldp) {
  const int cnt = *count;
  if (cnt <= 0) return;
  const int lane = threadIdx.x & 31;
  const int nslab = (cnt + kWideSlabH - 1) / kWideSlabH;
  const int64_t units = (int64_t)nslab * nitems;
  const int64_t nw = (int64_t)gridDim.x * (SPT / 32);
  for (int64_t w = (int64_t)blockIdx.x * (SPT / 32) + (threadIdx.x >> 5); w < units; w += nw) {
    const int slab = (int)(w / nitems), it = (int)(w - (int64_t)slab * nitems);
    const int k = slab * kWideSlabH + 4 * lane;   // this lane's starts k .. k + 3
    const bool on = k < cnt;                      // k + 3 < ldb whenever k < cnt (ldb a multiple of 16)
    const __half *B = Bt + k;
    const int4 head = __ldg(reinterpret_cast<const int4 *>(items + it));
    const int seg = head.z;
    for (int row = head.x; row < head.y; ++row) {
      const int64_t b = seg >= 0 ? items[it].nz0 : M.ptr[row];
      const int64_t e = seg >= 0 ? items[it].nz1 : M.ptr[row + 1];
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      for (int64_t base = b; base < e; base += 32) {
        const int m = (int)min((int64_t)32, e - base);
        const int jl = lane < m ? __ldg(M.col + base + lane) : 0;
        const float al = lane < m ? __ldg(M.val + base + lane) : 0.0f;
        int qq = 0;
        for (; qq + 8 <= m; qq += 8) {
          uint2 y[8];
          float a[8];
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            const int j = __shfl_sync(FULL, jl, qq + g);
            a[g] = __shfl_sync(FULL, al, qq + g);
            y[g] = on ? __ldg(reinterpret_cast<const uint2 *>(B + (int64_t)j * ldb)) : make_uint2(0u, 0u);
          }
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            const float2 lo = half2_bits(y[g].x), hi = half2_bits(y[g].y);
            acc[0] = fmaf(a[g], lo.x, acc[0]);
            acc[1] = fmaf(a[g], lo.y, acc[1]);
            acc[2] = fmaf(a[g], hi.x, acc[2]);
            acc[3] = fmaf(a[g], hi.y, acc[3]);
          }
        }
        for (; qq < m; ++qq) {
          const int j = __shfl_sync(FULL, jl, qq);
          const float a = __shfl_sync(FULL, al, qq);
          const uint2 y = on ? __ldg(reinterpret_cast<const uint2 *>(B + (int64_t)j * ldb)) : make_uint2(0u, 0u);
          const float2 lo = half2_bits(y.x), hi = half2_bits(y.y);
          acc[0] = fmaf(a, lo.x, acc[0]);
          acc[1] = fmaf(a, lo.y, acc[1]);
          acc[2] = fmaf(a, hi.x, acc[2]);
          acc[3] = fmaf(a, hi.y, acc[3]);
        }
      }
      if (on) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (k + t >= cnt) break;
          if (seg >= 0) part[(int64_t)seg * ldp + k + t] = acc[t];
          else out[(int64_t)(list ? list[k + t] : k + t) * ldo + row] = acc[t];
        }
      }
    }
  }
}

cudaError_t launch_spmm_h(SpMat M, const SpPlan &P, const float *Y, int64_t ldy, int len, const int *list,
                          const int *count, int rmax, void *Bt, int ldb16, float *out, int64_t ldo, float *part,
                          int ldp, int sms, cudaStream_t st) {
  __half *B = static_cast<__half *>(Bt);
  const dim3 pgrid((unsigned)((len + 31) / 32), (unsigned)((rmax + 31) / 32));
  k_pack_t_h<<<pgrid, dim3(32, 8), 0, st>>>(Y, ldy, len, list, count, B, ldb16);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (P.nitems > 0) {
    const bool wide = rmax > 32;
    const int64_t units = (int64_t)P.nitems * (wide ? (rmax + kWideSlabH - 1) / kWideSlabH : 1);
    const int64_t want = (units + SPT / 32 - 1) / (SPT / 32);
    const int blocks = (int)(want < sms * 8 ? want : sms * 8);
    if (wide)
      k_spmm_wide_h<<<blocks, SPT, 0, st>>>(M, P.items, P.nitems, B, ldb16, count, list, out, ldo, part, ldp);
    else if (rmax <= 16)
      k_spmm_h<1><<<blocks, SPT, 0, st>>>(M, P.items, P.nitems, B, ldb16, count, list, out, ldo, part, ldp);
    else
      k_spmm_h<2><<<blocks, SPT, 0, st>>>(M, P.items, P.nitems, B, ldb16, count, list, out, ldo, part, ldp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (P.nlong > 0) {
    k_spmm_fix<<<P.nlong, 256, 0, st>>>(P.longs, part, ldp, count, nullptr, list, out, ldo);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

// grid (ceil(n / SCH), r): u = A x for start c over x's support (A^T by rows = A by columns),
// for the starts the gather serves (active, swept at least once)
__global__ void __launch_bounds__(256) k_spmv_support(SpMat AT, int n, const int *__restrict__ sup_idx,
                                                      const float *__restrict__ sup_val, int cap, StartState s,
                                                      float *__restrict__ U, int64_t ldu,
                                                      const int *__restrict__ gate) {
  if (*gate == 0) return;
  const int c = blockIdx.y;
  if (s.status[c] != ST_ACTIVE) return;
  if (s.iters[c] == 0) return;   // a start not swept yet has a dense x: the product by rows
  __shared__ float us[SCH];
  __shared__ int64_t lo[256], hi[256];
  __shared__ float xv[256];
  const int base = blockIdx.x * SCH;
  const int rows = min(SCH, n - base);
  for (int i = threadIdx.x; i < SCH; i += 256) us[i] = 0.0f;
  const int nnz = s.nnz[c];
  const int *gi = sup_idx + (int64_t)c * cap;
  const float *gv = sup_val + (int64_t)c * cap;
  for (int t0 = 0; t0 < nnz; t0 += 256) {
    __syncthreads();
    if (t0 + (int)threadIdx.x < nnz) {
      const int j = gi[t0 + threadIdx.x];
      xv[threadIdx.x] = gv[t0 + threadIdx.x];
      const int64_t b = lower_bound_col(AT.col, AT.ptr[j], AT.ptr[j + 1], base);
      lo[threadIdx.x] = b;
      hi[threadIdx.x] = lower_bound_col(AT.col, b, AT.ptr[j + 1], base + rows);
    }
    __syncthreads();
    const int m = min(256, nnz - t0);
    for (int q = 0; q < m; ++q) {
      // the rows of one column are distinct: no two threads update the same u_i
      const float x = xv[q];
      for (int64_t k = lo[q] + threadIdx.x; k < hi[q]; k += 256) {
        const int i = __ldg(AT.col + k) - base;
        us[i] = fmaf(x, __ldg(AT.val + k), us[i]);
      }
      __syncthreads();
    }
  }
  __syncthreads();
  float *u = U + (int64_t)c * ldu + base;
  for (int i = threadIdx.x; i < rows; i += 256) u[i] = us[i];
}

cudaError_t launch_spmv_support(SpMat AT, int n, const int *sup_idx, const float *sup_val, int cap, StartState s,
                                int r, float *U, int64_t ldu, const int *gate, cudaStream_t st) {
  const dim3 grid((unsigned)((n + SCH - 1) / SCH), (unsigned)r);
  k_spmv_support<<<grid, 256, 0, st>>>(AT, n, sup_idx, sup_val, cap, s, U, ldu, gate);
  return cudaGetLastError();
}

// grid (ceil(n / 256), ceil(count / 8)): rows [256 b, 256 b + 256) of u = A x for the starts
// 8 g .. 8 g + 7, whose x are packed start-fastest in Bt (one 32-byte sector per entry for the 8),
// a warp per 32 rows.  Each lane keeps a compensated FP32-pair sum per start over a strided subset
// of the row; the lanes' pairs are added in a fixed butterfly in pair arithmetic, and so are the
// warp's sums of |u_i| and u_i^2 over its rows (GB300 issues FP64 at a small fraction of the FP32
// rate, so no FP64 runs per row).  Per CTA and start the warps' sums are added in warp order, in
// FP64, into partials[(c * nchunks + b) * 2 + {0, 1}].
// u_i -= sum_q coef[q] W[q, i] in pair arithmetic (coef in FP64, split into two floats)
__device__ __forceinline__ void lowrank_sub(F32Pair &u, const double *__restrict__ coef, const float *__restrict__ W,
                                            int64_t ldw, int k, int i) {
  for (int q = 0; q < k; ++q) {
    const float w = W[(int64_t)q * ldw + i];
    const float ch = (float)coef[q];
    const float cl = (float)(coef[q] - (double)ch);
    f32pair_fma(u, -ch, w);
    f32pair_fma(u, -cl, w);
  }
}

__global__ void __launch_bounds__(256) k_fin_csr(SpMat A, const float *__restrict__ Bt, int ldb, int count,
                                                 const int *__restrict__ nnz, int cap, float *__restrict__ U,
                                                 int64_t ldu, double *__restrict__ partials, const double *__restrict__ coef,
                                                 const float *__restrict__ W, int64_t ldw, int kdef) {
  __shared__ double red[8][8][2];
  const int b = blockIdx.x, c0 = blockIdx.y * 8;
  const int nc = min(8, count - c0);
  if (nnz) {   // starts whose support the column scatter serves are done there
    bool any = false;
    for (int g = 0; g < nc; ++g) any |= nnz[c0 + g] > cap;
    if (!any) return;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float *B = Bt + c0;
  F32Pair l1[8], l2[8];
  for (int q = 0; q < 32; ++q) {
    const int i = b * 256 + w * 32 + q;
    if (i >= A.rows) break;
    F32Pair acc[8];
    for (int64_t k = A.ptr[i] + lane; k < A.ptr[i + 1]; k += 32) {
      const float a = A.val[k];
      float xs[8];
      ldg8(B + (int64_t)A.col[k] * ldb, xs);
#pragma unroll
      for (int g = 0; g < 8; ++g) f32pair_fma(acc[g], a, xs[g]);
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      F32Pair t = acc[g];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        F32Pair other;
        other.hi = __shfl_xor_sync(FULL, t.hi, o);
        other.lo = __shfl_xor_sync(FULL, t.lo, o);
        t = f32pair_add(t, other);
      }
      // every lane now holds u_i (of A x; then of A_k x after deflation)
      if (kdef > 0 && g < nc) lowrank_sub(t, coef + (int64_t)(c0 + g) * kdef, W, ldw, kdef, i);
      if (lane == 0 && g < nc && !(nnz && nnz[c0 + g] <= cap)) U[(int64_t)(c0 + g) * ldu + i] = __fadd_rn(t.hi, t.lo);
      l1[g] = f32pair_add(l1[g], f32pair_abs(t));
      l2[g] = f32pair_add(l2[g], f32pair_sq(t));
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      red[w][g][0] = f32pair_value(l1[g]);
      red[w][g][1] = f32pair_value(l2[g]);
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < nc && !(nnz && nnz[c0 + threadIdx.x] <= cap)) {
    const int g = threadIdx.x;
    double s1 = 0.0, s2 = 0.0;
    for (int ww = 0; ww < 8; ++ww) {
      s1 += red[ww][g][0];
      s2 += red[ww][g][1];
    }
    double *o = partials + ((int64_t)(c0 + g) * gridDim.x + b) * 2;
    o[0] = s1;
    o[1] = s2;
  }
}

// grid (ceil(n / 256), count): rows [256 b, 256 b + 256) of u = A x for start c over its support
// (at most cap entries), from A by columns: each thread owns one row's compensated FP32-pair sum,
// the support's columns are added one at a time in support order (the products of one column go
// to distinct rows).  |u_i| and u_i^2 are summed over the CTA in pair arithmetic and written, as
// FP64, to partials like k_fin_csr's.
__global__ void __launch_bounds__(256) k_fin_support(SpMat AT, const int *__restrict__ sup_idx,
                                                     const float *__restrict__ sup_val, int ldsup,
                                                     const int *__restrict__ nnz, int cap, float *__restrict__ U,
                                                     int64_t ldu, double *__restrict__ partials,
                                                     const double *__restrict__ coef, const float *__restrict__ W,
                                                     int64_t ldw, int kdef) {
  __shared__ float us_hi[256], us_lo[256];
  __shared__ int64_t lo_s[256], hi_s[256];
  __shared__ float xv[256];
  __shared__ double red[8][2];
  const int b = blockIdx.x, c = blockIdx.y;
  const int m = nnz[c];
  if (m > cap) return;            // the rows' kernel serves this start
  const int base = b * 256, rows = min(256, AT.cols - base);
  us_hi[threadIdx.x] = 0.0f;
  us_lo[threadIdx.x] = 0.0f;
  for (int t0 = 0; t0 < m; t0 += 256) {
    __syncthreads();
    if (t0 + (int)threadIdx.x < m) {
      const int j = sup_idx[(int64_t)c * ldsup + t0 + threadIdx.x];
      xv[threadIdx.x] = sup_val[(int64_t)c * ldsup + t0 + threadIdx.x];
      const int64_t lo = lower_bound_col(AT.col, AT.ptr[j], AT.ptr[j + 1], base);
      lo_s[threadIdx.x] = lo;
      hi_s[threadIdx.x] = lower_bound_col(AT.col, lo, AT.ptr[j + 1], base + rows);
    }
    __syncthreads();
    const int mm = min(256, m - t0);
    for (int q = 0; q < mm; ++q) {
      // a column holds at most one entry per row: at most 256 entries in this chunk
      const int64_t k = lo_s[q] + threadIdx.x;
      if (k < hi_s[q]) {
        const int i = AT.col[k] - base;
        F32Pair s;
        s.hi = us_hi[i];
        s.lo = us_lo[i];
        f32pair_fma(s, xv[q], AT.val[k]);
        us_hi[i] = s.hi;
        us_lo[i] = s.lo;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  F32Pair u;
  u.hi = us_hi[threadIdx.x];
  u.lo = us_lo[threadIdx.x];
  if (kdef > 0 && (int)threadIdx.x < rows) lowrank_sub(u, coef + (int64_t)c * kdef, W, ldw, kdef, base + threadIdx.x);
  if ((int)threadIdx.x < rows) U[(int64_t)c * ldu + base + threadIdx.x] = __fadd_rn(u.hi, u.lo);
  F32Pair a1 = f32pair_abs(u), a2 = f32pair_sq(u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    F32Pair t1, t2;
    t1.hi = __shfl_xor_sync(FULL, a1.hi, o);
    t1.lo = __shfl_xor_sync(FULL, a1.lo, o);
    t2.hi = __shfl_xor_sync(FULL, a2.hi, o);
    t2.lo = __shfl_xor_sync(FULL, a2.lo, o);
    a1 = f32pair_add(a1, t1);
    a2 = f32pair_add(a2, t2);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[w][0] = f32pair_value(a1);
    red[w][1] = f32pair_value(a2);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s1 = 0.0, s2 = 0.0;
    for (int ww = 0; ww < 8; ++ww) {
      s1 += red[ww][0];
      s2 += red[ww][1];
    }
    double *o = partials + ((int64_t)c * gridDim.x + b) * 2;
    o[0] = s1;
    o[1] = s2;
  }
}

// starts with at most kSpSupportCap nonzeros (when their support lists are given): the column
// scatter; the others by rows, in groups of at most ldb (the packed operand's width)
cudaError_t launch_fin_csr(SpMat A, SpMat AT, const float *X, int64_t ldx, int count, const int *nnz,
                           const int *sup_idx, const float *sup_val, int ldsup, float *Bt, int ldb, float *U,
                           int64_t ldu, double *partials, LowRank L, cudaStream_t st) {
  const int nchunks = (A.rows + 255) / 256;
  const int cap = sup_idx ? kSpSupportCap : -1;
  if (sup_idx) {
    k_fin_support<<<dim3((unsigned)nchunks, (unsigned)count), 256, 0, st>>>(AT, sup_idx, sup_val, ldsup, nnz, cap, U,
                                                                              ldu, partials, L.coef, L.W, L.ldw, L.k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  for (int c0 = 0; c0 < count; c0 += ldb) {
    const int m = count - c0 < ldb ? count - c0 : ldb;
    cudaError_t e = launch_pack_t(X + (int64_t)c0 * ldx, ldx, A.cols, nullptr, nullptr, nullptr, m, Bt, ldb, st);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)nchunks, (unsigned)((m + 7) / 8));
    k_fin_csr<<<grid, 256, 0, st>>>(A, Bt, ldb, m, sup_idx ? nnz + c0 : nullptr, cap, U + (int64_t)c0 * ldu, ldu,
                                    partials + (int64_t)c0 * nchunks * 2, L.k > 0 ? L.coef + (int64_t)c0 * L.k : nullptr,
                                    L.W, L.ldw, L.k);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------- low-rank deflation
// grid (count): coef[list[b] * k + q] = z_q^T x_c for the start c = list[b] (or b), in FP64 from
// compensated FP32-pair sums per thread
__global__ void __launch_bounds__(256) k_lowrank_coef(const float *__restrict__ X, int64_t ldx, int p,
                                                      const int *__restrict__ list, const int *__restrict__ count,
                                                      int count_host, const float *__restrict__ Z, int64_t ldz, int k,
                                                      double *__restrict__ coef) {
  __shared__ double red[32];
  const int cnt = count ? *count : count_host;
  if ((int)blockIdx.x >= cnt) return;
  const int c = list ? list[blockIdx.x] : (int)blockIdx.x;
  const float *x = X + (int64_t)c * ldx;
  for (int q = 0; q < k; ++q) {
    const float *z = Z + (int64_t)q * ldz;
    F32Pair s;
    for (int j = threadIdx.x; j < p; j += blockDim.x) f32pair_fma(s, z[j], x[j]);
    const double t = block_sum_d(f32pair_value(s), red);
    if (threadIdx.x == 0) coef[(int64_t)c * k + q] = t;
    __syncthreads();
  }
}

// grid (ceil(len / 1024), count): out[c][i] -= sum_q coef[c * k + q] B[q][i] (u -= W (Z^T x) with
// B = W, v -= Z (W^T y) with B = Z), FP32
__global__ void __launch_bounds__(256) k_lowrank_axpy(float *__restrict__ out, int64_t ldo, int len,
                                                      const int *__restrict__ list, const int *__restrict__ count,
                                                      int count_host, const float *__restrict__ B, int64_t ldb_, int k,
                                                      const double *__restrict__ coef) {
  const int cnt = count ? *count : count_host;
  if ((int)blockIdx.y >= cnt) return;
  const int c = list ? list[blockIdx.y] : (int)blockIdx.y;
  float *o = out + (int64_t)c * ldo;
  for (int i = blockIdx.x * 1024 + threadIdx.x; i < min(len, (int)(blockIdx.x + 1) * 1024); i += blockDim.x) {
    float v = o[i];
    for (int q = 0; q < k; ++q) v = fmaf(-(float)coef[(int64_t)c * k + q], B[(int64_t)q * ldb_ + i], v);
    o[i] = v;
  }
}

cudaError_t launch_lowrank_coef(const float *src, int64_t lds, int src_len, const int *list, const int *count,
                                int rmax, const float *Cdot, int64_t ldc, int k, double *coef, cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  k_lowrank_coef<<<rmax, 256, 0, st>>>(src, lds, src_len, list, count, rmax, Cdot, ldc, k, coef);
  return cudaGetLastError();
}

cudaError_t launch_lowrank(const float *src, int64_t lds, int src_len, float *out, int64_t ldo, int out_len,
                           const int *list, const int *count, int rmax, const float *Cdot, int64_t ldc,
                           const float *B, int64_t ldb_, int k, double *coef, cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  cudaError_t e = launch_lowrank_coef(src, lds, src_len, list, count, rmax, Cdot, ldc, k, coef, st);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((out_len + 1023) / 1024), (unsigned)rmax);
  k_lowrank_axpy<<<grid, 256, 0, st>>>(out, ldo, out_len, list, count, rmax, B, ldb_, k, coef);
  return cudaGetLastError();
}

// one CTA: z = x / ||x||_2 (||x|| in FP64); *bad = 1 when x = 0 (z left as is)
__global__ void __launch_bounds__(1024) k_unit(const float *__restrict__ x, int p, float *__restrict__ z, int *bad) {
  __shared__ double red[32];
  double s = 0.0;
  for (int j = threadIdx.x; j < p; j += blockDim.x) s += (double)x[j] * (double)x[j];
  const double nrm = sqrt(block_sum_d(s, red));
  if (!(nrm > 0.0)) {
    if (threadIdx.x == 0) *bad = 1;
    return;
  }
  const double inv = 1.0 / nrm;
  for (int j = threadIdx.x; j < p; j += blockDim.x) z[j] = (float)((double)x[j] * inv);
}

cudaError_t launch_unit(const float *x, int p, float *z, int *bad, cudaStream_t st) {
  k_unit<<<1, 1024, 0, st>>>(x, p, z, bad);
  return cudaGetLastError();
}

}  // namespace spca
