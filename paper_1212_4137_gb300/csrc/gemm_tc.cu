// gemm_tc.cu -- the two contractions of an AM sweep (u = A x, v = A^T y; Algorithm 2) on the
// 5th-generation tensor cores (tcgen05, sm_103a): TMA loads into 128B-swizzled shared memory,
// one elected thread issues tcgen05.mma with the accumulator in TMEM, four epilogue warps read
// TMEM back with tcgen05.ld and store the result transposed (one start per output row).
//
// FP32-class accuracy from FP16 tensor cores: every FP32 operand is stored as two FP16 planes of
// a power-of-two scaled copy (hi = fp16(s a), lo = fp16(s a - hi): 22 significant bits; see
// kPlanes in spca_internal.cuh).  A product sum a.b is then the sum over plane pairs (i, j) of
// a_i . b_j, each product exact; the pairs hi.hi, hi.lo and lo.hi carry everything above the
// 2^-21 relative level (3 products for two general operands, 2 when b is +-1 and has one
// plane).  The tensor core's accumulation truncates, so the error grows with the number of MMA
// steps into one accumulator: the hi x hi product goes to its own TMEM accumulator and the
// correction products (2^-11 smaller) to a second one; the epilogue adds the two with FP32
// round-to-nearest and undoes the scales (a power of two).  Measured with three BF16 planes on
// GB300 against FP64 (K = 8192, relative to sum |a_k b_k|): one accumulator for all products
// 3.5e-6, the hi x hi product alone 7.6e-7.
//
//   D[m, c] = sum_{(i,j) in pairs} sum_k P_i[m, k] Q_j[c, k]      out[c * ldo + m] = D[m, c]
//
// P (M x K) and Q (N x K) are K-contiguous FP16 planes; plane i of P starts at row i * M_alloc.
// Two kernels: the CTA-pair kernel (k_gemm_tc2, 256-row tiles, persistent stream-K) whenever
// the output has two or more 128-row tiles, and a single-CTA kernel (k_gemm_tc, 128-row tiles,
// one CTA per output tile, no cluster) for a lone M tile and for handles that share the
// device with other solves.  Every CTA loads its own operand tiles; no load is multicast.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstdint>

#include "block_util.cuh"
#include "spca_internal.cuh"

namespace spca {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_THREADS = 192;           // warp 0 TMA + TMEM alloc, warp 1 MMA, warps 2-5 epilogue
// the CTA-pair kernel: warp 0 TMA + TMEM alloc, warp 1 MMA, warps 2-9 epilogue (two warps per TMEM
// lane quarter, each holding the running sum of 128 of the tile's 256 columns in registers)
constexpr int TC2_THREADS = 320;
constexpr int TC2_EPI_WARPS = 8;
// bounded waits: the limit is a launch argument (2 s unless a handle sets a shorter one), after
// which a kernel records SPCA_E_TIMEOUT and winds down; loads still in flight then get at most
// TC_DRAIN_NS to land before the CTA exits
constexpr uint64_t TC_DRAIN_NS = 1000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the phase with the given parity; false (and *err set) after wait_ns nanoseconds, or
// at once when another thread of the CTA has given up (*abort_flag)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err, volatile int *abort_flag,
                                          uint64_t wait_ns) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > wait_ns) {
      *abort_flag = 1;
      if (err) atomicExch(err, SPCA_E_TIMEOUT);
      return false;
    }
  }
}
// the same without error reporting, for the clean-up after a wait gave up
__device__ __forceinline__ bool mbar_wait_quiet(uint32_t bar, uint32_t parity, uint64_t wait_ns) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try(bar, parity))
    if (globaltimer() - t0 > wait_ns) return false;
  return true;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
// shared-memory matrix descriptor: K-major rows of BK bf16 (BK = 64: 128B swizzle; BK = 32:
// 64B swizzle), 8-row core groups 8 * 2 * BK bytes apart
template <int BK>
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);             // start address
  d |= (uint64_t)1 << 16;                                // leading byte offset (unused here)
  d |= (uint64_t)((8 * 2 * BK) >> 4) << 32;             // stride byte offset: 8 rows
  d |= (uint64_t)1 << 46;                                // descriptor version (tcgen05)
  d |= (uint64_t)(BK == 64 ? 2 : 4) << 61;               // swizzle: 128B or 64B
  return d;
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// instruction descriptor, kind::f16: D f32 (bit 4), A and B f16 (format 0 in bits 7-9 and
// 10-12), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

}  // namespace

template <int BN, int NA, int NB, int STAGES, int TC_BK>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmQ, int M, int N,
              int kblocks, const int *__restrict__ k_dev, TcPairs pairs, float *__restrict__ out, int64_t ldo,
              const float *__restrict__ row_inv, const float *__restrict__ col_inv, float q_inv,
              const int *__restrict__ gate, const int *__restrict__ n_dev, const int *__restrict__ col_map,
              int *err, uint64_t wait_ns, int ntn_launch) {
  constexpr uint32_t A_BYTES = TC_BM * TC_BK * 2;       // 16 KB per P plane tile
  constexpr uint32_t B_BYTES = BN * TC_BK * 2;          // 16 KB (BN = 128) per Q plane tile
  constexpr uint32_t STAGE_BYTES = NA * A_BYTES + NB * B_BYTES;
  // four FP32 accumulators of BN columns x 128 lanes: the hi x hi product of K-block kb goes to
  // accumulator kb mod nmain (three of them, four without correction products) and the
  // corrections to the last one.  The tensor core's accumulation truncates, so its error grows
  // with the steps into one accumulator and with the accumulator's magnitude: spreading the
  // main product over three accumulators cuts that error threefold.
  constexpr uint32_t TMEM_COLS = 4 * BN;
  static_assert(TMEM_COLS <= 512, "TMEM columns");

  extern __shared__ __align__(1024) uint8_t dsmem[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], accum_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  if (gate && *gate == 0) return;   // uniform over the grid: the contraction is not needed
  if (n_dev) N = *n_dev;            // columns (active starts) known only on the device
  if (k_dev) kblocks = (*k_dev + TC_BK - 1) / TC_BK;   // contraction length known only on the device
  if (kblocks <= 0) return;
  // one linear grid over the output tiles, N tiles fastest (CTAs sharing a P tile run together);
  // ntn_launch = the N tiles the grid was sized for (N may be smaller when read from the device)
  const int tn = (int)(blockIdx.x % (unsigned)ntn_launch), tm = (int)(blockIdx.x / (unsigned)ntn_launch);
  if (tn * BN >= N) return;   // uniform over the CTA

  uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = tm * TC_BM, n0 = tn * BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);             // this CTA's MMA commit
    }
    mbar_init(smem_u32(&accum_bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  // the producer counts the stages whose loads it issued, the MMA issuer the stages it consumed:
  // after a timed-out wait the producer waits (bounded) for the loads still in flight
  __shared__ int issued, consumed;
  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------------- TMA producer
    int kb = 0;
    for (; kb < kblocks; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, err, &abort_flag, wait_ns)) break;
      const uint32_t fb = smem_u32(&full_bar[s]);
      mbar_expect_tx(fb, STAGE_BYTES);
      uint8_t *st = tiles + (size_t)s * STAGE_BYTES;
#pragma unroll
      for (int a = 0; a < NA; ++a) tma_load_3d(smem_u32(st + a * A_BYTES), &tmP, kb * TC_BK, m0, a, fb);
#pragma unroll
      for (int b = 0; b < NB; ++b)
        tma_load_3d(smem_u32(st + NA * A_BYTES + b * B_BYTES), &tmQ, kb * TC_BK, n0, b, fb);
    }
    issued = kb;
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------------- MMA issuer
    constexpr uint32_t idesc = idesc_f16(TC_BM, BN);
    const int nmain = pairs.first_corr >= 0 ? 3 : 4;
    bool ok = true;
    int kb = 0;
    for (; kb < kblocks && ok; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(smem_u32(&full_bar[s]), ph, err, &abort_flag, wait_ns)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = smem_u32(tiles + (size_t)s * STAGE_BYTES);
      for (int q = 0; q < pairs.n; ++q) {
        const uint32_t a_base = st + pairs.a[q] * A_BYTES;
        const uint32_t b_base = st + NA * A_BYTES + pairs.b[q] * B_BYTES;
        const bool main = (pairs.a[q] | pairs.b[q]) == 0;   // hi x hi -> accumulator kb mod nmain
        const uint32_t d = tmem + (uint32_t)BN * (main ? (uint32_t)(kb % nmain) : 3u);
        const bool first = main ? (kb < nmain && q == pairs.first_main) : (kb == 0 && q == pairs.first_corr);
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk) {
          mma_bf16(d, sw_desc<TC_BK>(a_base + kk * 32), sw_desc<TC_BK>(b_base + kk * 32), idesc,
                   (first && kk == 0) ? 0u : 1u);
        }
      }
      mma_commit(smem_u32(&empty_bar[s]));   // frees the stage once these MMAs have read it
    }
    consumed = kb;
    // the accumulator is complete (after a wait gave up: the MMAs issued so far are done, which
    // the clean-up below waits for before it frees TMEM)
    mma_commit(smem_u32(&accum_bar));
  } else if (warp >= 2) {
    // ---------------------------------------------------------------- epilogue (TMEM -> HBM)
    const int quad = warp & 3;                 // TMEM lanes 32*quad .. 32*quad+31
    // tcgen05.ld is warp-collective: take the barrier result uniformly over the warp
    const bool ready = __all_sync(0xffffffffu, mbar_wait(smem_u32(&accum_bar), 0, err, &abort_flag, wait_ns) &&
                                                   !abort_flag);
    if (ready) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = m0 + quad * 32 + lane;
      const int nmain = pairs.first_corr >= 0 ? 3 : 4;
      const int nused = kblocks < nmain ? kblocks : nmain;   // main accumulators written
#pragma unroll 1
      for (int cb = 0; cb < BN / 32; ++cb) {
        float v[32], w[32];
        const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(cb * 32);
        tmem_ld32(ta, v);
        // the main accumulators in order, then the corrections
        for (int i = 1; i < nused; ++i) {
          tmem_ld32(ta + (uint32_t)(i * BN), w);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += w[j];
        }
        if (pairs.first_corr >= 0) {
          tmem_ld32(ta + (uint32_t)(3 * BN), w);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += w[j];
        }
        if (row < M) {
          const float sc = (row_inv ? row_inv[row] : 1.0f) * q_inv;   // powers of two
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + cb * 32 + j;
            if (col < N)
              out[(int64_t)(col_map ? col_map[col] : col) * ldo + row] = v[j] * sc * (col_inv ? col_inv[col] : 1.0f);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (abort_flag && threadIdx.x == 0) {
    // a wait gave up: the MMAs issued so far may still run, and the loads of the stages issued
    // but not consumed may still be landing in this CTA's shared memory; wait for both (bounded)
    // before TMEM is freed and the CTA exits
    mbar_wait_quiet(smem_u32(&accum_bar), 0, wait_ns);
    for (int kb = consumed; kb < issued; ++kb)
      mbar_wait_quiet(smem_u32(&full_bar[kb % STAGES]), (uint32_t)(kb / STAGES) & 1u, TC_DRAIN_NS);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------------------------- CTA-pair variant
// A cluster of two CTAs computes 256 x BN tiles with tcgen05 .cta_group::2: each CTA loads its
// own 128 rows of the P planes and its half (BN/2 rows) of the Q planes to the same shared-memory
// offsets; the leader (cluster rank 0) issues the MMAs with M = 256, which read both CTAs' shared
// memory, and each CTA's TMEM receives its own 128 rows of D.  The peer's loads complete on the
// leader's full barrier; the leader's commits free the stage and signal the accumulator in both
// CTAs.  Per SM this doubles the MMA work per loaded byte of Q and per pipeline stage compared
// with the single-CTA tile.
//
// Persistent stream-K schedule: the grid is S resident pairs ("slots"); the T tiles x KB K-blocks
// of the product are numbered tile-major (M pair fastest within an N column of tiles, so that
// slots running at the same time share P rows in L2), and slot j takes the units
// [j W / S, (j + 1) W / S), W = T KB -- an equal share whatever T is, so no wave runs part-empty.
// A slot walks its range as segments, one per tile it touches; a segment is a whole tile (its
// epilogue writes the output), the first K-blocks of a tile (the slot then owns the tile), or a
// later part of one (the slot's first segment: it writes the partial to its workspace slot and
// publishes a flag, set to `epoch` = 1; the flags are zeroed before every launch).  An owner's
// part is the last segment of its range, so by then the later
// parts, which other slots compute first, are mostly done: it waits for their flags (bounded),
// adds them in slot order and writes the tile.  The TMEM accumulators are reused from segment to
// segment: the epilogue of both CTAs releases them before the leader's next MMA.
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                                 uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar_cluster)
      : "memory");
}
__device__ __forceinline__ void mma_bf16_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// the same for 8-bit operands (kind::f8f6f4; with A and B both E4M3 the instruction descriptor's
// format fields are 0, as for f16: K = 32 elements, 32 bytes, per instruction)
__device__ __forceinline__ void mma_f8_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
      ::"r"(bar), "h"((uint16_t)3)
      : "memory");
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_s32(uint32_t addr_cluster, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr_cluster), "r"(v) : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// order earlier generic-proxy writes of a tensor map in global memory before tensor loads through it
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_local(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// split points of a tile's K range for the main accumulator: the multiples of `piece` K-blocks
// (piece <= 0: none)
__device__ __forceinline__ bool is_split(int kb, int piece) { return piece > 0 && kb > 0 && kb % piece == 0; }
// the smallest split point above kb (INT32_MAX when there is none)
__device__ __forceinline__ int next_split(int kb, int piece) {
  return piece > 0 ? (kb / piece + 1) * piece : 0x7fffffff;
}
// split points strictly inside (kb0, kb1)
__device__ __forceinline__ int splits_inside(int kb0, int kb1, int piece) {
  return piece > 0 && kb1 - 1 > kb0 ? (kb1 - 1) / piece - kb0 / piece : 0;
}

struct SkRange {   // slot j's share of the W units: [u0, u1)
  long long W;
  int S;
  __device__ long long start(int j) const { return (long long)j * W / S; }
};

// F8: operands in FP8 E4M3 (one byte each; a K-block of 128 elements keeps the 128-byte swizzled
// rows of the FP16 layout, so the stage layout, descriptors and the 32-byte MMA steps are the same)
template <int BN, int NA, int NB, int STAGES, bool F8 = false>
__global__ void __launch_bounds__(TC2_THREADS, 1)
    k_gemm_tc2(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmQ, int M, int N,
               int kblocks, const int *__restrict__ k_dev, TcPairs pairs, float *__restrict__ out, int64_t ldo,
               const float *__restrict__ row_inv, const float *__restrict__ col_inv, float q_inv,
               const int *__restrict__ gate, const int *__restrict__ n_dev, const int *__restrict__ col_map,
               int *err, float *__restrict__ ws, int *__restrict__ flags, int epoch, int wait_epoch,
               uint64_t wait_ns, int piece) {
  constexpr int ES = F8 ? 1 : 2;                        // bytes per element
  constexpr int BK = 128 / ES;                          // elements per K-block: 128-byte rows
  constexpr uint32_t A_BYTES = TC_BM * BK * ES;         // this CTA's 128 rows of one P plane
  constexpr uint32_t B_BYTES = (BN / 2) * BK * ES;      // this CTA's half of one Q plane
  constexpr uint32_t STAGE_BYTES = NA * A_BYTES + NB * B_BYTES;
  constexpr uint32_t TMEM_COLS = 2 * BN;

  extern __shared__ __align__(1024) uint8_t dsmem[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], accum_bar, tmem_empty_bar, mma_done_bar,
      part_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  // clean-up bookkeeping: stages whose loads this CTA issued, stages the leader's MMAs consumed,
  // and (in the leader) the peer's issued count and abort flag, written by the peer
  __shared__ int issued, consumed, peer_issued, peer_abort;

  const uint32_t rank = cluster_rank();   // 0: leader (even M tile of the pair), 1: peer
  const int slot = (int)(blockIdx.x >> 1), S = (int)(gridDim.x >> 1);
  if (gate && *gate == 0) return;         // uniform over the grid
  if (n_dev) N = *n_dev;
  const int KB = k_dev ? (*k_dev + BK - 1) / BK : kblocks;
  const int pm = ((M + TC_BM - 1) / TC_BM + 1) / 2;   // pairs of 128-row tiles along M
  const int ntn = (N + BN - 1) / BN;
  SkRange R{(long long)pm * ntn * (KB > 0 ? KB : 0), S};
  if (R.W <= 0) return;
  const long long u0 = R.start(slot), u1 = R.start(slot + 1);
  if (u0 >= u1) return;                   // an empty share (uniform over the pair)

  uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&accum_bar), 1);
    mbar_init(smem_u32(&tmem_empty_bar), 2 * TC2_EPI_WARPS);   // the epilogue warps of both CTAs
    mbar_init(smem_u32(&mma_done_bar), 1);     // the leader's last commit: every MMA done
    mbar_init(smem_u32(&part_bar), TC2_EPI_WARPS);   // the epilogue warps wrote a stream-K part (one per slot)
    abort_flag = 0;
    issued = consumed = peer_issued = peer_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  cluster_sync_all();   // both CTAs' barriers and TMEM exist before any load or MMA reaches them
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  // segment iteration shared by the three roles: tile t, K-blocks [kb0, kb1)
  auto next_seg = [&](long long &u, long long &t, int &kb0, int &kb1) {
    t = u / KB;
    kb0 = (int)(u - t * KB);
    const long long e = (t + 1) * KB < u1 ? (t + 1) * KB : u1;
    kb1 = (int)(e - t * KB);
    u = e;
  };

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------------- TMA producer (both CTAs)
    uint32_t it = 0;
    bool ok = true;
    for (long long u = u0; u < u1 && ok;) {
      long long t;
      int kb0, kb1;
      next_seg(u, t, kb0, kb1);
      const int m0 = (2 * (int)(t % pm) + (int)rank) * TC_BM, n0 = (int)(t / pm) * BN;
      for (int kb = kb0; kb < kb1; ++kb, ++it) {
        const int s = (int)(it % STAGES);
        const uint32_t ph = (it / STAGES) & 1u;
        if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, err, &abort_flag, wait_ns)) { ok = false; break; }
        const uint32_t own = smem_u32(&full_bar[s]);
        const uint32_t fb = rank == 0 ? own : map_to_rank(own, 0);   // the leader's full barrier
        if (rank == 0) mbar_expect_tx(own, 2 * STAGE_BYTES);         // both CTAs' bytes
        uint8_t *st = tiles + (size_t)s * STAGE_BYTES;
#pragma unroll
        for (int a = 0; a < NA; ++a) tma_load_3d_pair(smem_u32(st + a * A_BYTES), &tmP, kb * BK, m0, a, fb);
#pragma unroll
        for (int b = 0; b < NB; ++b)
          tma_load_3d_pair(smem_u32(st + NA * A_BYTES + b * B_BYTES), &tmQ, kb * BK, n0 + (int)rank * (BN / 2), b,
                           fb);
      }
    }
    issued = (int)it;
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---------------------------------------------------------------- MMA issuer (leader)
    // Every commit to accum_bar is one "drain": the epilogues of both CTAs read the accumulators
    // (the main one alone at a split point, main and corrections at the end of a segment) and
    // release them on tmem_empty_bar; drain d's release is phase d of that barrier.
    // At a split point of the tile's K range the main accumulator is drained into the epilogue's
    // registers and restarted, so that no main accumulation spans more than `piece` K-blocks (the
    // accumulation truncates, and its error grows with the steps into one accumulator and with
    // the accumulator's magnitude).  To keep the tensor pipe busy meanwhile, the last STAGES
    // stages before a split issue their main products only; once the drain is committed their
    // correction products follow (into their own accumulator) while the epilogue reads the main
    // one.  Each accumulator still receives its products in K order, so the result does not
    // depend on the timing.
    constexpr uint32_t idesc = idesc_f16(2 * TC_BM, BN);
    const bool has_corr = pairs.first_corr >= 0;
    uint32_t it = 0, nd = 0;
    bool ok = true;
    auto issue = [&](uint32_t st, bool do_main, bool do_corr, bool main_first, bool corr_first) {
      for (int q = 0; q < pairs.n; ++q) {
        const bool main = (pairs.a[q] | pairs.b[q]) == 0;
        if (main ? !do_main : !do_corr) continue;
        const uint32_t a_base = st + pairs.a[q] * A_BYTES;
        const uint32_t b_base = st + NA * A_BYTES + pairs.b[q] * B_BYTES;
        const uint32_t d = tmem + (main ? 0u : (uint32_t)BN);
        const bool first = main ? (main_first && q == pairs.first_main) : (corr_first && q == pairs.first_corr);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {   // 32 bytes of K per instruction
          if (F8)
            mma_f8_pair(d, sw_desc<64>(a_base + kk * 32), sw_desc<64>(b_base + kk * 32), idesc,
                        (first && kk == 0) ? 0u : 1u);
          else
            mma_bf16_pair(d, sw_desc<64>(a_base + kk * 32), sw_desc<64>(b_base + kk * 32), idesc,
                          (first && kk == 0) ? 0u : 1u);
        }
      }
    };
    uint32_t pend_st[STAGES];   // stages whose correction products wait for the next split's drain
    int pend_s[STAGES];
    bool pend_first[STAGES];
    for (long long u = u0; u < u1 && ok;) {
      long long t;
      int kb0, kb1;
      next_seg(u, t, kb0, kb1);
      // the epilogues of both CTAs have read the previous drain
      if (nd > 0 && !mbar_wait(smem_u32(&tmem_empty_bar), (nd - 1) & 1u, err, &abort_flag, wait_ns)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      bool main_first = true;
      int npend = 0;
      int nxt = has_corr ? next_split(kb0, piece) : 0x7fffffff;   // the next split point after kb0
      for (int kb = kb0; kb < kb1; ++kb, ++it) {
        const int s = (int)(it % STAGES);
        const uint32_t ph = (it / STAGES) & 1u;
        if (!mbar_wait(smem_u32(&full_bar[s]), ph, err, &abort_flag, wait_ns)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = smem_u32(tiles + (size_t)s * STAGE_BYTES);
        if (nxt < kb1 && nxt - kb <= STAGES) {
          // one of the last STAGES stages before a split: main products now, corrections later
          issue(st, true, false, main_first, false);
          pend_st[npend] = st;
          pend_s[npend] = s;
          pend_first[npend] = kb == kb0;
          ++npend;
        } else {
          issue(st, true, true, main_first, kb == kb0);
          mma_commit_pair(smem_u32(&empty_bar[s]));   // frees stage s in both CTAs
        }
        main_first = false;
        if (kb + 1 == nxt && nxt < kb1) {
          // the main piece ends here: drain nd reads the main accumulator alone
          mma_commit_pair(smem_u32(&accum_bar));
          ++nd;
          for (int q = 0; q < npend; ++q) {
            issue(pend_st[q], false, true, false, pend_first[q]);
            mma_commit_pair(smem_u32(&empty_bar[pend_s[q]]));
          }
          npend = 0;
          if (!mbar_wait(smem_u32(&tmem_empty_bar), (nd - 1) & 1u, err, &abort_flag, wait_ns)) {
            ok = false;
            ++it;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          main_first = true;
          nxt = next_split(nxt, piece);
        }
      }
      if (ok) {
        mma_commit_pair(smem_u32(&accum_bar));      // drain nd: the segment's result
        ++nd;
      }
    }
    consumed = (int)it;
    // every MMA issued so far is done when this completes (in both CTAs): the clean-up waits for
    // it before TMEM is freed
    mma_commit_pair(smem_u32(&mma_done_bar));
  } else if (warp >= 2) {
    // ---------------------------------------------------------------- epilogue (own 128 rows)
    // warp w reads TMEM lanes 32 (w mod 4) .. + 31 (rows of this CTA's half of the tile) and
    // columns 128 h .. 128 h + 127, h = (w - 2) / 4; the running sum of those 128 columns of its
    // row stays in registers, so a split drain costs four TMEM loads and no memory traffic
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const uint32_t tmem_empty_leader = map_to_rank(smem_u32(&tmem_empty_bar), 0);
    const int row_l = quad * 32 + lane, cbase = half * 128;
    const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)cbase;
    const bool has_corr = pairs.first_corr >= 0;
    uint32_t nd = 0;
    bool ok = true;
    for (long long u = u0; u < u1 && ok;) {
      float acc[128];
      long long t;
      int kb0, kb1;
      next_seg(u, t, kb0, kb1);
      const bool owner = kb0 == 0 && kb1 < KB, contrib = kb0 > 0;
      const int m0 = (2 * (int)(t % pm) + (int)rank) * TC_BM, n0 = (int)(t / pm) * BN;
      // the split drains of the main accumulator inside this segment, then the segment's result:
      // acc = ((main_1 + main_2) + ... + main_last) + corrections, in that order
      const int nsplit = has_corr ? splits_inside(kb0, kb1, piece) : 0;
      for (int d = 0; d <= nsplit && ok; ++d) {
        ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&accum_bar), nd & 1u, err, &abort_flag, wait_ns));
        ++nd;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (d == 0) {
#pragma unroll
          for (int cb = 0; cb < 8; ++cb) {
            float v[16];
            tmem_ld16(tbase + (uint32_t)(cb * 16), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[cb * 16 + j] = v[j];
          }
        } else {
#pragma unroll
          for (int cb = 0; cb < 8; ++cb) {
            float v[16];
            tmem_ld16(tbase + (uint32_t)(cb * 16), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[cb * 16 + j] += v[j];
          }
        }
        if (d == nsplit && has_corr) {
#pragma unroll
          for (int cb = 0; cb < 8; ++cb) {
            float v[16];
            tmem_ld16(tbase + (uint32_t)BN + (uint32_t)(cb * 16), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[cb * 16 + j] += v[j];
          }
        }
        // accumulators read: release them to the leader's next MMA
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(tmem_empty_leader);
      }
      if (!ok) break;
      // an owner waits for the later parts of its tile (slots slot+1, slot+2, ...)
      int jlast = slot;
      if (owner) {
        const long long tend = (t + 1) * KB;
        while (jlast + 1 < S && R.start(jlast + 1) < tend) ++jlast;
        if (lane == 0) {
          for (int j = slot + 1; j <= jlast && ok; ++j) {
            if (R.start(j) >= R.start(j + 1)) continue;   // empty share: no part
            const int *fl = flags + (j * 2 + (int)rank);
            if (ld_acquire(fl) == wait_epoch) continue;
            const uint64_t t0 = globaltimer();
            while (ld_acquire(fl) != wait_epoch) {
              if (abort_flag || globaltimer() - t0 > wait_ns) {
                abort_flag = 1;
                if (err) atomicExch(err, SPCA_E_TIMEOUT);
                ok = false;
                break;
              }
            }
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        __syncwarp();
      }
      const int row = m0 + row_l;
      float *mine = ws + ((int64_t)slot * 2 + rank) * BN * TC_BM;
      if (contrib) {
#pragma unroll
        for (int c = 0; c < 128; ++c) __stcg(mine + (int64_t)(cbase + c) * TC_BM + row_l, acc[c]);
        // this part of the tile is in the workspace: each warp signals its rows, then warp 2
        // publishes the part once all of them have (a bounded wait on an mbarrier rather than a
        // named barrier, so that a warp that gave up cannot leave the others blocked)
        __syncwarp();
        if (lane == 0) mbar_arrive_local(smem_u32(&part_bar));
        if (warp == 2 && lane == 0 && mbar_wait(smem_u32(&part_bar), 0, err, &abort_flag, wait_ns)) {
          __threadfence();
          st_release(flags + (slot * 2 + (int)rank), epoch);
        }
        continue;
      }
      if (owner && ok) {
        for (int jj = slot + 1; jj <= jlast; ++jj) {
          if (R.start(jj) >= R.start(jj + 1)) continue;
          const float *part = ws + ((int64_t)jj * 2 + rank) * BN * TC_BM + (int64_t)cbase * TC_BM + row_l;
#pragma unroll
          for (int cb = 0; cb < 8; ++cb) {   // 16 loads in flight at a time
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __ldcg(part + (int64_t)(cb * 16 + j) * TC_BM);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[cb * 16 + j] += v[j];
            __syncwarp();
          }
        }
      }
      // (row < M differs between the lanes of the last row tile: no warp-wide operation below)
      if (row < M && ok) {
        const float sc = (row_inv ? row_inv[row] : 1.0f) * q_inv;   // powers of two
#pragma unroll
        for (int c = 0; c < 128; ++c) {
          const int col = n0 + cbase + c;
          if (col < N)
            out[(int64_t)(col_map ? col_map[col] : col) * ldo + row] = acc[c] * sc * (col_inv ? col_inv[col] : 1.0f);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (rank == 1 && threadIdx.x == 0) {
    // the peer's loads complete on the leader's barriers: tell the leader how far they went
    st_cluster_s32(map_to_rank(smem_u32(&peer_issued), 0), issued);
    st_cluster_s32(map_to_rank(smem_u32(&peer_abort), 0), abort_flag);
  }
  cluster_sync_all();
  if (threadIdx.x == 0) {
    // the leader's MMAs into this CTA's TMEM (and out of its shared memory) are done
    mbar_wait_quiet(smem_u32(&mma_done_bar), 0, wait_ns);
    if (rank == 0 && (abort_flag || peer_abort)) {
      // a wait gave up: stages loaded but not consumed may still be landing in either CTA's
      // shared memory.  Each such stage has one open phase on the leader's full barrier; a stage
      // only the peer loaded is armed here for the peer's bytes.  Bounded waits.
      const int top = issued > peer_issued ? issued : peer_issued;
      for (int q = consumed; q < top; ++q) {
        const uint32_t fb = smem_u32(&full_bar[q % STAGES]);
        if (q >= issued) mbar_expect_tx(fb, STAGE_BYTES);
        mbar_wait_quiet(fb, (uint32_t)(q / STAGES) & 1u, TC_DRAIN_NS);
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
  cluster_sync_all();   // the peer leaves only after the leader's clean-up
}

// ---------------------------------------------------------------------- planes
// dst plane t (t < nplanes) of element e: the t-th FP16 piece of the scaled src (hi, lo)
__global__ void k_split_planes(const float *__restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                               __half *__restrict__ dst, int64_t ldd, int64_t plane_stride, int nplanes,
                               const float *__restrict__ row_scale, float scale, const int *__restrict__ gate,
                               const int *__restrict__ rows_dev, const int *__restrict__ row_map) {
  if (gate && *gate == 0) return;
  if (rows_dev) rows = *rows_dev;
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e - r * cols;
    // s a is exact (a power of two); hi = fp16(s a); the remainder s a - hi is exact in FP32
    const float a = src[(row_map ? (int64_t)row_map[r] : r) * lds + c] * (row_scale ? row_scale[r] : scale);
    const __half hi = __float2half_rn(a);
    const int64_t o = r * ldd + c;
    dst[o] = hi;
    if (nplanes > 1) dst[o + plane_stride] = __float2half_rn(a - __half2float(hi));
  }
}

cudaError_t launch_split_planes(const float *src, int64_t rows, int64_t cols, int64_t lds, void *dst,
                                int64_t ldd, int64_t plane_stride, int nplanes, const float *row_scale,
                                float scale, const int *gate, const int *rows_dev, const int *row_map,
                                cudaStream_t st) {
  // a grid-stride loop over 4 CTAs per SM: when the gate is off the launch costs only that many
  // early exits
  k_split_planes<<<608, 256, 0, st>>>(src, rows, cols, lds, static_cast<__half *>(dst), ldd, plane_stride, nplanes,
                                      row_scale, scale, gate, rows_dev, row_map);
  return cudaGetLastError();
}

// dst row r = E4M3(src row row_map[r] (identity when null) x row_scale[r] x mul (x mul alone
// when row_scale is null)), saturating at the largest finite E4M3; r < rows (*rows_dev when given);
// gated
__global__ void k_split_f8(const float *__restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                           uint8_t *__restrict__ dst, int64_t ldd, const float *__restrict__ row_scale, float mul,
                           const int *__restrict__ gate, const int *__restrict__ rows_dev,
                           const int *__restrict__ row_map) {
  if (gate && *gate == 0) return;
  if (rows_dev) rows = *rows_dev;
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e - r * cols;
    const float a = src[(row_map ? (int64_t)row_map[r] : r) * lds + c] * ((row_scale ? row_scale[r] : 1.0f) * mul);
    dst[r * ldd + c] = __nv_cvt_float_to_fp8(a, __NV_SATFINITE, __NV_E4M3);
  }
}

cudaError_t launch_split_f8(const float *src, int64_t rows, int64_t cols, int64_t lds, uint8_t *dst, int64_t ldd,
                            const float *row_scale, float mul, const int *gate, const int *rows_dev,
                            const int *row_map, cudaStream_t st) {
  k_split_f8<<<608, 256, 0, st>>>(src, rows, cols, lds, dst, ldd, row_scale, mul, gate, rows_dev, row_map);
  return cudaGetLastError();
}

// dst[i] = src[i] x mul, i < n (the inverse scales of a copy scaled by 1 / mul); gated
__global__ void k_scale_copy(const float *__restrict__ src, int n, float mul, float *__restrict__ dst,
                             const int *__restrict__ gate) {
  if (gate && *gate == 0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i] * mul;
}

cudaError_t launch_scale_copy(const float *src, int n, float mul, float *dst, const int *gate, cudaStream_t st) {
  k_scale_copy<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, st>>>(src, n, mul, dst, gate);
  return cudaGetLastError();
}

// one CTA per row: scale = 2^(13 - floor(log2 max |row|)), so the scaled row's largest entry lies
// in [2^13, 2^14) (FP16's largest finite value is 65504); 1 for a zero row
__global__ void __launch_bounds__(256) k_row_scale(const float *__restrict__ src, int64_t cols, int64_t lds,
                                                   float *__restrict__ scale, float *__restrict__ inv,
                                                   const int *__restrict__ gate, const int *__restrict__ rows_dev,
                                                   const int *__restrict__ row_map) {
  __shared__ unsigned red[32];
  if (gate && *gate == 0) return;
  if (rows_dev && (int)blockIdx.x >= *rows_dev) return;
  const float *row = src + (row_map ? (int64_t)row_map[blockIdx.x] : (int64_t)blockIdx.x) * lds;
  unsigned mk = 0u;
  for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) mk = max(mk, __float_as_uint(fabsf(row[c])));
  const unsigned m = block_max_u(mk, red);
  if (threadIdx.x == 0) {
    int e = 0;
    if (m != 0u) {
      const float mx = __uint_as_float(m);
      e = 13 - ilogbf(mx);
      e = max(-120, min(120, e));
    }
    scale[blockIdx.x] = ldexpf(1.0f, e);
    inv[blockIdx.x] = ldexpf(1.0f, -e);
  }
}

cudaError_t launch_row_scales(const float *src, int64_t rows, int64_t cols, int64_t lds, float *scale, float *inv,
                              const int *gate, const int *rows_dev, const int *row_map, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  k_row_scale<<<(unsigned)rows, 256, 0, st>>>(src, cols, lds, scale, inv, gate, rows_dev, row_map);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------- host side
namespace {
// (function-local statics: initialised once, thread-safe, for handles used from several threads)
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}
}  // namespace

// 3-D map over `planes` FP16 planes of `rows` x `ld` (K-contiguous), box bk x box_rows x 1
cudaError_t make_plane_map(CUtensorMap *map, const void *base, int64_t rows, int64_t ld, int planes,
                           int box_rows, int bk) {
  auto enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * 2 * (cuuint64_t)rows};
  cuuint32_t box[3] = {(cuuint32_t)bk, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
// one FP8 (one byte per element) plane of rows x ld, box 128 x box_rows, 128-byte swizzle (ld a
// multiple of 16 bytes)
cudaError_t make_f8_map(CUtensorMap *map, const void *base, int64_t rows, int64_t ld, int box_rows) {
  auto enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  if (ld % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return cudaErrorInvalidValue;
  cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)rows, 1};
  cuuint64_t strides[2] = {(cuuint64_t)ld, (cuuint64_t)ld * (cuuint64_t)rows};
  cuuint32_t box[3] = {128, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void *>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_p_maps(PMaps *maps, const void *base, int64_t rows, int64_t ld, int planes) {
  return make_plane_map(&maps->m[0], base, rows, ld, planes, TC_BM, 64);
}

namespace {
template <int BN, int NA, int NB, int STAGES, int TC_BK>
cudaError_t launch_tc_impl(const PMaps &P, const CUtensorMap &Q, int M, int N, int K, const int *k_dev, TcPairs pairs,
                           float *out, int64_t ldo, const float *row_inv, const float *col_inv, float q_inv,
                           const int *gate, const int *n_dev, const int *col_map, int *err, uint64_t wait_ns,
                           cudaStream_t st) {
  constexpr int STAGE_BYTES = NA * TC_BM * TC_BK * 2 + NB * BN * TC_BK * 2;
  constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
  auto kern = k_gemm_tc<BN, NA, NB, STAGES, TC_BK>;
  static const cudaError_t configured = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  if (configured != cudaSuccess) return configured;
  // one CTA per 128 x BN output tile, N tiles fastest so that the CTAs reading one P tile run
  // together and share it through L2
  const int ntn = (N + BN - 1) / BN;
  const int64_t ctas = (int64_t)ntn * ((M + TC_BM - 1) / TC_BM);
  if (ctas < 1 || ctas > INT32_MAX) return cudaErrorInvalidValue;
  const int kblocks = (K + TC_BK - 1) / TC_BK;
  kern<<<(unsigned)ctas, TC_THREADS, SMEM, st>>>(P.m[0], Q, M, N, kblocks, k_dev, pairs, out, ldo, row_inv, col_inv,
                                                q_inv, gate, n_dev, col_map, err, wait_ns, ntn);
  return cudaGetLastError();
}
}  // namespace

namespace {
template <int BN, int NA, int NB, int STAGES, bool F8 = false>
cudaError_t launch_tc2_impl(const PMaps &P, const CUtensorMap &Q, int M, int N, int K, const int *k_dev,
                            TcPairs pairs, float *out, int64_t ldo, const float *row_inv, const float *col_inv,
                            float q_inv, const int *gate, const int *n_dev, const int *col_map, int *err,
                            const TcStreamK &sk, cudaStream_t st) {
  constexpr int ES = F8 ? 1 : 2;
  constexpr int BK = 128 / ES;
  constexpr int STAGE_BYTES = NA * TC_BM * BK * ES + NB * (BN / 2) * BK * ES;
  constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
  auto kern = k_gemm_tc2<BN, NA, NB, STAGES, F8>;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(TC2_THREADS);
  cfg.dynamicSmemBytes = SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // the slots must all be resident at once (owners wait for other slots' parts): as many pairs
  // as the device holds together, measured once per configuration
  static const int max_pairs = [&] {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM) != cudaSuccess) return 0;
    cudaLaunchConfig_t c = cfg;
    c.gridDim = dim3(2 * 64, 1);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &c) != cudaSuccess) return 0;
    return n;
  }();
  if (max_pairs < 1) return cudaErrorInvalidConfiguration;
  const int pm = ((M + TC_BM - 1) / TC_BM + 1) / 2, ntn = (N + BN - 1) / BN;
  const int kblocks = (K + BK - 1) / BK;
  const long long units = (long long)pm * ntn * kblocks;
  int S = max_pairs < sk.slots ? max_pairs : sk.slots;
  if (units < S) S = (int)(units > 0 ? units : 1);
  cfg.gridDim = dim3((unsigned)(2 * S), 1);
  // the flags of the parts start at 0 for every launch (a memset, so that a launch replayed from a
  // CUDA graph does not see the parts of the previous replay); a published part sets its flag to 1
  cudaError_t e = cudaMemsetAsync(sk.flags, 0, (size_t)2 * S * sizeof(int), st);
  if (e != cudaSuccess) return e;
  // the main product's K pieces: as even as possible, at most sk.piece_kb K-blocks each (with
  // correction products only: the leading-plane products need no FP32-class accuracy)
  int piece = 0;
  if (pairs.first_corr >= 0 && sk.piece_kb > 0 && kblocks > sk.piece_kb) {
    const int npieces = (kblocks + sk.piece_kb - 1) / sk.piece_kb;
    piece = (kblocks + npieces - 1) / npieces;
  }
  // parts are published with epoch 1; owners wait for sk.wait_epoch (1 unless a test asks for parts
  // that never come)
  return cudaLaunchKernelEx(&cfg, kern, P.m[0], Q, M, N, kblocks, k_dev, pairs, out, ldo, row_inv, col_inv, q_inv,
                            gate, n_dev, col_map, err, sk.ws, sk.flags, 1, sk.wait_epoch, sk.wait_ns, piece);
}
}  // namespace

// N width of the CTA-pair tile: 256 (512 TMEM columns: the hi x hi and the correction
// accumulators of 256 columns each) or 128; each CTA of a pair loads BN / 2 rows of Q, and the
// single-CTA tile used for a lone M tile is BN / 2 wide so that both read the same Q boxes
#ifndef SPCA_TC_PAIR_BN
#define SPCA_TC_PAIR_BN 256
#endif
constexpr int TC_PAIR_BN = SPCA_TC_PAIR_BN;
static_assert(TC_PAIR_BN == 128 || TC_PAIR_BN == 256, "pair tile width");

namespace {
// pipeline stages that fit in shared memory (227 KB per CTA, less 1 KB of alignment slack and
// 1 KB of barriers): na P planes of 128 x 64 plus nb Q planes of (BN / 2) x 64, FP16 -- the same
// per CTA for the pair tile and for the single-CTA tile; at most 8
constexpr int tc_stages(int na, int nb) {
  return (230400 / (na * TC_BM * 64 * 2 + nb * (TC_PAIR_BN / 2) * 64 * 2)) > 8
             ? 8
             : 230400 / (na * TC_BM * 64 * 2 + nb * (TC_PAIR_BN / 2) * 64 * 2);
}

// the single-CTA kernel: 128 x (BN / 2) tiles
cudaError_t launch_gemm_tc_single(const PMaps &P, int na, const CUtensorMap &Q, int nb, int M, int N, int K,
                                  const int *k_dev, TcPairs pairs, float *out, int64_t ldo, const float *row_inv,
                                  const float *col_inv, float q_inv, const int *gate, const int *n_dev,
                                  const int *col_map, int *err, uint64_t wait_ns, cudaStream_t st) {
  constexpr int BN1 = TC_PAIR_BN / 2;
  if (na == 2 && nb == 2)
    return launch_tc_impl<BN1, 2, 2, tc_stages(2, 2), 64>(P, Q, M, N, K, k_dev, pairs, out, ldo, row_inv, col_inv,
                                                          q_inv, gate, n_dev, col_map, err, wait_ns, st);
  if (na == 2 && nb == 1)
    return launch_tc_impl<BN1, 2, 1, tc_stages(2, 1), 64>(P, Q, M, N, K, k_dev, pairs, out, ldo, row_inv, col_inv,
                                                          q_inv, gate, n_dev, col_map, err, wait_ns, st);
  if (na == 1 && nb == 1)
    return launch_tc_impl<BN1, 1, 1, tc_stages(1, 1), 64>(P, Q, M, N, K, k_dev, pairs, out, ldo, row_inv, col_inv,
                                                          q_inv, gate, n_dev, col_map, err, wait_ns, st);
  return cudaErrorInvalidValue;
}
}  // namespace

// CTA pairs (256 x BN tiles, stream-K over the resident pairs) when there are at least two M
// tiles; one M tile runs on single CTAs
cudaError_t launch_gemm_tc(const PMaps &P, int na, const CUtensorMap &Q, int nb, int M, int N, int K,
                           const int *k_dev, TcPairs pairs, float *out, int64_t ldo, const float *row_inv,
                           const float *col_inv, float q_inv, const int *gate, const int *n_dev, const int *col_map,
                           int *err, const TcStreamK &sk, cudaStream_t st) {
  if (M <= TC_BM || !sk.ws || !sk.flags || sk.slots < 1)
    return launch_gemm_tc_single(P, na, Q, nb, M, N, K, k_dev, pairs, out, ldo, row_inv, col_inv, q_inv, gate,
                                 n_dev, col_map, err, sk.wait_ns, st);
  if (na == 2 && nb == 2)   // two general operands
    return launch_tc2_impl<TC_PAIR_BN, 2, 2, tc_stages(2, 2)>(P, Q, M, N, K, k_dev, pairs, out, ldo, row_inv,
                                                                col_inv, q_inv, gate, n_dev, col_map, err, sk, st);
  if (na == 2 && nb == 1)   // y = +-1
    return launch_tc2_impl<TC_PAIR_BN, 2, 1, tc_stages(2, 1)>(P, Q, M, N, K, k_dev, pairs, out, ldo, row_inv,
                                                                col_inv, q_inv, gate, n_dev, col_map, err, sk, st);
  if (na == 1 && nb == 1)   // the leading planes only (low-precision sweeps)
    return launch_tc2_impl<TC_PAIR_BN, 1, 1, tc_stages(1, 1)>(P, Q, M, N, K, k_dev, pairs, out, ldo, row_inv,
                                                                col_inv, q_inv, gate, n_dev, col_map, err, sk, st);
  return cudaErrorInvalidValue;
}

// Q-operand boxes: BN / 2 rows (half of a pair tile, or a whole single-CTA tile)
cudaError_t launch_gemm_tc_f8(const PMaps &P, const CUtensorMap &Q, int M, int N, int K, const int *k_dev,
                              float *out, int64_t ldo, const float *row_inv, const float *col_inv, float q_inv,
                              const int *gate, const int *n_dev, const int *col_map, int *err, const TcStreamK &sk,
                              cudaStream_t st) {
  if (M <= TC_BM || !sk.ws || !sk.flags || sk.slots < 1) return cudaErrorInvalidValue;   // pair kernel only
  TcPairs hi{};
  hi.n = 1;
  hi.first_main = 0;
  hi.first_corr = -1;
  return launch_tc2_impl<TC_PAIR_BN, 1, 1, tc_stages(1, 1), true>(P, Q, M, N, K, k_dev, hi, out, ldo, row_inv,
                                                                  col_inv, q_inv, gate, n_dev, col_map, err, sk, st);
}

// ---------------------------------------------------------------------- grouped contraction
// One persistent launch over the tiles of many independent contractions (one per problem of a
// group): task i computes out_i[map(c) * ldo + m] = (row_inv[m] q_inv col_inv[c]) sum_q sum_k
// P_i,a_q[m, k] Q_i,b_q[c, k] for m < M_i and c < *n_dev_i, like launch_gemm_tc, each with its own
// tensor maps (held in global memory), K, plane products and output.  The tiles (128 x BN) of all
// tasks form one list (tile t = task tiles[t].x, local tile tiles[t].y: M tile local / nt, N tile
// local % nt) in an order the host chooses: tasks on the same matrix interleaved by M tile, so
// that the CTAs running at the same time read each tile of the shared matrix once from DRAM and
// then from L2; tasks by falling K, so that the round-robin below balances.  CTA b takes tiles
// b, b + G, b + 2G, ...  Every role of a CTA walks the same tile sequence, so no tile index is
// exchanged between them.
// TMEM: NBUF = 512 / (4 BN) buffers of four accumulators (BN = 64: two buffers, so a tile's
// epilogue overlaps the next tile's MMAs).  The hi x hi product of K-block kb goes to accumulator
// kb mod 3 and the correction products to the fourth (FP32-class accuracy, see k_gemm_tc).
// LOWP: every task takes the leading planes only (one P plane, one Q plane, one product: the
// sweeps of resident 16-bit matrices, whose inputs carry 11 significant bits); one accumulator per
// tile, so tiles up to 256 columns wide still get two TMEM buffers.
template <int BN, int STAGES, bool LOWP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_grouped(const GTask *__restrict__ tasks, const int2 *__restrict__ tile_list, int total_tiles, int *err,
                   uint64_t wait_ns) {
  constexpr int NA = LOWP ? 1 : 2, NBMAX = LOWP ? 1 : 2, NACC = LOWP ? 1 : 4;
  constexpr uint32_t A_BYTES = TC_BM * 64 * 2;            // 16 KB per P plane tile
  constexpr uint32_t B_BYTES = BN * 64 * 2;               // one Q plane tile (BN rows)
  constexpr uint32_t STAGE_BYTES = NA * A_BYTES + NBMAX * B_BYTES;
  constexpr int NBUF = 512 / (NACC * BN);
  constexpr uint32_t TMEM_COLS = 512;
  static_assert(NBUF >= 1 && NBUF * NACC * BN <= (int)TMEM_COLS, "TMEM");

  extern __shared__ __align__(1024) uint8_t dsmem[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], accum_bar[NBUF], tmem_empty_bar[NBUF],
      mma_done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int issued, consumed;

  const int G = gridDim.x;
  if ((int)blockIdx.x >= total_tiles) return;
  uint8_t *tiles = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(smem_u32(&accum_bar[b]), 1);
      mbar_init(smem_u32(&tmem_empty_bar[b]), 4);   // the four epilogue warps
    }
    mbar_init(smem_u32(&mma_done_bar), 1);            // the MMA issuer's last commit
    abort_flag = 0;
    issued = consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  // tile t -> (task, M tile, N tile); false when the tile lies past the task's active columns
  auto locate = [&](int t, int &ti, int &m0, int &n0, int &N) -> bool {
    const int2 e = tile_list[t];
    ti = e.x;
    const GTask &T = tasks[ti];
    const int local = e.y;
    const int tn = local % T.nt, tm = local / T.nt;
    m0 = tm * TC_BM;
    n0 = tn * BN;
    N = T.n_dev ? *T.n_dev : T.nmax;
    return n0 < N && T.kblocks > 0;
  };

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------------- TMA producer
    uint32_t it = 0;
    bool ok = true;
    int last_task = -1;
    for (int t = blockIdx.x; t < total_tiles && ok; t += G) {
      int ti, m0, n0, N;
      if (!locate(t, ti, m0, n0, N)) continue;
      const GTask &T = tasks[ti];
      if (ti != last_task) {
        // the maps live in global memory and may have been rewritten since an earlier launch:
        // order those writes before this CTA's tensor loads through them
        tensormap_acquire(T.pmap);
        tensormap_acquire(T.qmap);
        last_task = ti;
      }
      const uint32_t bytes = (uint32_t)T.na * A_BYTES + (uint32_t)T.nb * B_BYTES;
      for (int kb = 0; kb < T.kblocks; ++kb, ++it) {
        const int s = (int)(it % STAGES);
        const uint32_t ph = (it / STAGES) & 1u;
        if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, err, &abort_flag, wait_ns)) { ok = false; break; }
        const uint32_t fb = smem_u32(&full_bar[s]);
        mbar_expect_tx(fb, bytes);
        uint8_t *st = tiles + (size_t)s * STAGE_BYTES;
        for (int a = 0; a < T.na; ++a) tma_load_3d(smem_u32(st + a * A_BYTES), T.pmap, kb * 64, m0, a, fb);
        for (int b = 0; b < T.nb; ++b)
#pragma unroll
          for (int h = 0; h < BN / 64; ++h)
            tma_load_3d(smem_u32(st + NA * A_BYTES + b * B_BYTES + h * 64 * 128), T.qmap, kb * 64, n0 + 64 * h, b,
                        fb);
      }
    }
    issued = (int)it;
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------------- MMA issuer
    constexpr uint32_t idesc = idesc_f16(TC_BM, BN);
    uint32_t it = 0, ntile = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < total_tiles && ok; t += G) {
      int ti, m0, n0, N;
      if (!locate(t, ti, m0, n0, N)) continue;
      const GTask &T = tasks[ti];
      const TcPairs pairs = T.pairs;
      const int b = (int)(ntile % NBUF);
      // this buffer's previous tile has been read by the epilogue
      if (ntile >= (uint32_t)NBUF &&
          !mbar_wait(smem_u32(&tmem_empty_bar[b]), ((ntile / NBUF) - 1) & 1u, err, &abort_flag, wait_ns)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dbase = tmem + (uint32_t)(b * NACC * BN);
      for (int kb = 0; kb < T.kblocks; ++kb, ++it) {
        const int s = (int)(it % STAGES);
        const uint32_t ph = (it / STAGES) & 1u;
        if (!mbar_wait(smem_u32(&full_bar[s]), ph, err, &abort_flag, wait_ns)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = smem_u32(tiles + (size_t)s * STAGE_BYTES);
        for (int q = 0; q < pairs.n; ++q) {
          const uint32_t a_base = st + pairs.a[q] * A_BYTES;
          const uint32_t b_base = st + NA * A_BYTES + pairs.b[q] * B_BYTES;
          const bool main = (pairs.a[q] | pairs.b[q]) == 0;
          // a leading-planes task (one product) accumulates in one accumulator in either variant,
          // so that its sums are the same whichever variant the group runs
          const bool one = LOWP || pairs.n == 1;
          const uint32_t d = one ? dbase : dbase + (uint32_t)BN * (main ? (uint32_t)(kb % 3) : 3u);
          const bool first = one ? (kb == 0 && q == 0)
                                 : main ? (kb < 3 && q == pairs.first_main) : (kb == 0 && q == pairs.first_corr);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_bf16(d, sw_desc<64>(a_base + kk * 32), sw_desc<64>(b_base + kk * 32), idesc,
                     (first && kk == 0) ? 0u : 1u);
        }
        mma_commit(smem_u32(&empty_bar[s]));
      }
      if (!ok) break;
      mma_commit(smem_u32(&accum_bar[b]));
      ++ntile;
    }
    consumed = (int)it;
    mma_commit(smem_u32(&mma_done_bar));   // completes once every MMA issued so far is done
  } else if (warp >= 2) {
    // ---------------------------------------------------------------- epilogue
    const int quad = warp & 3;
    const int row_l = quad * 32 + lane;
    uint32_t ntile = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < total_tiles && ok; t += G) {
      int ti, m0, n0, N;
      if (!locate(t, ti, m0, n0, N)) continue;
      const GTask &T = tasks[ti];
      const int b = (int)(ntile % NBUF);
      ok = __all_sync(0xffffffffu,
                      mbar_wait(smem_u32(&accum_bar[b]), (ntile / NBUF) & 1u, err, &abort_flag, wait_ns) &&
                          !abort_flag);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int nused = LOWP || T.pairs.n == 1 ? 1 : T.kblocks < 3 ? T.kblocks : 3;
      const bool corr = !LOWP && T.pairs.first_corr >= 0;
      const int row = m0 + row_l;
      const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * NACC * BN);
#pragma unroll 1
      for (int cb = 0; cb < BN / 32; ++cb) {
        float v[32], w[32];
        tmem_ld32(tb + (uint32_t)(cb * 32), v);
        for (int i = 1; i < nused; ++i) {
          tmem_ld32(tb + (uint32_t)(i * BN + cb * 32), w);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += w[j];
        }
        if (corr) {
          tmem_ld32(tb + (uint32_t)(3 * BN + cb * 32), w);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += w[j];
        }
        if (row < T.M) {
          const float sc = (T.row_inv ? T.row_inv[row] : 1.0f) * T.q_inv;   // powers of two
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + cb * 32 + j;
            if (col < N)
              T.out[(int64_t)(T.col_map ? T.col_map[col] : col) * T.ldo + row] =
                  v[j] * sc * (T.col_inv ? T.col_inv[col] : 1.0f);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_local(smem_u32(&tmem_empty_bar[b]));
      ++ntile;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    // every MMA is done before TMEM is freed; after a wait gave up, the loads issued but not
    // consumed also land (bounded) before the CTA exits
    mbar_wait_quiet(smem_u32(&mma_done_bar), 0, wait_ns);
    if (abort_flag)
      for (int q = consumed; q < issued; ++q)
        mbar_wait_quiet(smem_u32(&full_bar[q % STAGES]), (uint32_t)(q / STAGES) & 1u, TC_DRAIN_NS);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

namespace {
template <int BN, int STAGES, bool LOWP>
cudaError_t launch_grouped_impl(const GTask *tasks, const int2 *tile_list, int total_tiles, int grid, int *err,
                                uint64_t wait_ns, cudaStream_t st) {
  constexpr int NP = LOWP ? 1 : 2;   // planes of each operand a stage holds
  constexpr int STAGE_BYTES = NP * TC_BM * 64 * 2 + NP * BN * 64 * 2;
  constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
  static_assert(SMEM <= 227 * 1024, "shared memory");
  auto kern = k_gemm_grouped<BN, STAGES, LOWP>;
  static const cudaError_t configured = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  if (configured != cudaSuccess) return configured;
  kern<<<grid, TC_THREADS, SMEM, st>>>(tasks, tile_list, total_tiles, err, wait_ns);
  return cudaGetLastError();
}
}  // namespace

bool grouped_config_ok(int bn, int stages, bool lowp) {
  if (lowp) return (bn == 64 || bn == 128 || bn == 256) && stages >= 2 && stages <= 4;
  return (bn == 64 && (stages == 2 || stages == 3 || stages == 4)) || (bn == 128 && (stages == 2 || stages == 3));
}

cudaError_t launch_gemm_grouped(const GTask *tasks, const int2 *tile_list, int total_tiles, int bn, int stages,
                                bool lowp, int sms, int *err, uint64_t wait_ns, cudaStream_t st) {
  if (total_tiles < 1) return cudaSuccess;   // nothing to contract
  const int grid = total_tiles < sms ? total_tiles : sms;
#define SPCA_GROUPED(B, S, L) \
  if (bn == B && stages == S && lowp == L) \
    return launch_grouped_impl<B, S, L>(tasks, tile_list, total_tiles, grid, err, wait_ns, st);
  SPCA_GROUPED(64, 2, false)
  SPCA_GROUPED(64, 3, false)
  SPCA_GROUPED(64, 4, false)
  SPCA_GROUPED(128, 2, false)
  SPCA_GROUPED(128, 3, false)
  SPCA_GROUPED(64, 2, true)
  SPCA_GROUPED(64, 3, true)
  SPCA_GROUPED(64, 4, true)
  SPCA_GROUPED(128, 2, true)
  SPCA_GROUPED(128, 3, true)
  SPCA_GROUPED(128, 4, true)
  SPCA_GROUPED(256, 2, true)
  SPCA_GROUPED(256, 3, true)
  SPCA_GROUPED(256, 4, true)
#undef SPCA_GROUPED
  return cudaErrorInvalidValue;
}

int tc_box_rows(int nb) { (void)nb; return TC_PAIR_BN / 2; }

// workspace of the stream-K schedule: one 256 x BN FP32 part per pair slot
int64_t tc_sk_floats_per_slot() { return (int64_t)2 * TC_BM * TC_PAIR_BN; }
int tc_bk(int nb) { (void)nb; return 64; }

}  // namespace spca
