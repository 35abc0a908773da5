// spca_internal.cuh -- shared declarations of the CUDA side of libspca (sm_103a).
//
// Layout in HBM (per handle):
//   A32   n x ldA  FP32, row-major copy of A             (dense y-side contraction, SIMT)
//   AT32  p x ldAT FP32, A transposed (column-major A)   (x-side contraction, sparse gathers,
//                                                          FP64 objective)
// Per solve (workspace, r starts, one vector per row):
//   X  r x ldX   current iterates x        U  r x ldU  u = A x
//   Y  r x ldU   y-step result             V  r x ldX  v = A^T y
//   support lists (idx, val) r x cap, per-start scalars, control words.
// Leading dimensions are padded to a multiple of 8 elements and the pad is kept at zero,
// so contraction kernels need no K-tail guards.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/spca.h"

namespace spca {

constexpr int kPad = 8;  // leading dimensions are multiples of 8 elements
inline int64_t pad_ld(int64_t m) { return (m + kPad - 1) / kPad * kPad; }

// formulation predicates (Table 1 numbering)
__host__ __device__ inline bool is_l1_var(int f) { return (f % 2) == 0; }
__host__ __device__ inline bool is_pen(int f) { return f >= 5; }
__host__ __device__ inline bool uses_T(int f) { return f == 1 || f == 2; }
__host__ __device__ inline bool uses_lam(int f) { return f == 3 || f == 4; }
__host__ __device__ inline bool uses_U(int f) { return f == 5 || f == 6; }
__host__ __device__ inline bool uses_V(int f) { return f == 7 || f == 8; }

constexpr int ST_ACTIVE = -1;  // device-side: still iterating (host sees SPCA_ST_* only)

// control words, one set per sweep parity (double-buffered so that the x-step of sweep k
// writes the flags the contractions of sweep k+1 read)
// Every path decision of the next sweep's u = A x is made on the device, so the host can queue
// sweeps ahead without reading anything back: exactly one of need_dense, use_union and
// use_gather is set for the next sweep.
struct Ctrl {
  int active;      // starts still iterating after this sweep
  int need_dense;  // some active start has more nonzeros than the sparse paths hold: dense u
  int use_union;   // u over the union of the supports (tensor cores)
  int use_gather;  // u by the per-start support gather
  int kunion;      // size of the union of the active starts' supports
  int err;         // kernel-reported error code (0 = none)
  int sum_nnz;     // sum of the active starts' support sizes (bounds the union; saturates)
  int max_nnz;     // largest active support
  int n_retire;    // on-the-fly replacement: slots whose start stopped in this sweep ...
  int n_new;       // ... and how many of them took a new start (dense x: the next u = A x of
                   // those slots is the dense contraction over them)
};

// per-start state of one solve (device arrays, r each)
struct StartState {
  int *status;      // ST_ACTIVE or SPCA_ST_*
  int *iters;       // sweeps performed
  int *nnz;         // nonzeros of x
  double *F;        // F of the last sweep
  double *F_prev;   // F of the sweep before
  double *gamma;    // gamma (penalty forms, in the units of Table 1)
  float *thr;       // the same threshold in |v| units, as a float the kernels compare with
  double *f;        // Table 1 objective (finalise)
  double *ev;       // explained variance (finalise)
  float *tprev;     // last sweep's x-step threshold in |v| units (0: none); seeds the
                    // candidate filter of the next x-step
  int *xfast;       // nonzero when the candidate x-step finished the start in this sweep (its guess)
};

struct XstepArgs {
  int form;
  int p;
  double s;
  int calibrate;       // apply the Section 4.1 gamma rule in this sweep
  int per_start_thr;   // penalty threshold from StartState (frozen after calibration)
  float thr_fixed;     // otherwise: the fixed threshold in |v| units ...
  double gamma_fixed;  // ... and gamma in Table 1 units
  int stop_test;       // stopping rule allowed in this sweep
  double tol;
  int max_iter;
  int cap;             // capacity of each support list (entries per start)
  int sparse_cap;      // larger supports make the next sweep use the dense u = A x
  // per-start schedule (solves): the switches above follow each start's own sweep count it
  // (StartState::iters, counted by the y-step): calibrate while it <= calib_sweeps in the
  // gamma-targeting mode, the frozen per-start threshold after, and the stopping rule from
  // it >= max(2, calib_sweeps + 1, lowp_sweeps + 2) when stop_enabled
  int schedule;
  int target;
  int calib_sweeps;
  int lowp_sweeps;
  int stop_enabled;
};

// the x-step switches of start c under XstepArgs::schedule (else as given)
__device__ inline XstepArgs xstep_switches(XstepArgs a, const int *iters, int c) {
  if (!a.schedule) return a;
  const int it = iters[c];
  a.calibrate = a.target && it <= a.calib_sweeps;
  a.per_start_thr = a.target && it > a.calib_sweeps;
  a.stop_test = a.stop_enabled && it >= 2 && it >= a.calib_sweeps + 1 && it >= a.lowp_sweeps + 2;
  return a;
}

// ---------------------------------------------------------------- kernels (launchers)
// each returns cudaGetLastError() of its launch(es)
cudaError_t launch_transpose_f32(const float *src, int64_t rows, int64_t cols, int64_t lds,
                                 float *dst, int64_t ldd, cudaStream_t st);
cudaError_t launch_convert_f64_f32(const double *src, int64_t rows, int64_t cols, int64_t lds,
                                   float *dst, int64_t ldd, cudaStream_t st);
cudaError_t launch_copy_f32(const float *src, int64_t rows, int64_t cols, int64_t lds,
                            float *dst, int64_t ldd, cudaStream_t st);
cudaError_t launch_check_finite(const float *a, int64_t rows, int64_t cols, int64_t ld,
                                int *flag, cudaStream_t st);

// a1: x^(0) = g / ||g||_2 (g from x0, or seeded normals when x0 == nullptr); resets the
// per-start state (gamma0 = the fixed gamma of a penalty form, else 0).  Row c of X is start c;
// with slot_list, the k-th listed slot (k < *count) takes start slot_start[slot] (its row of x0,
// or normal numbers start * p + j of the seeded stream)
cudaError_t launch_start_init(const float *x0, int64_t ld0, uint64_t seed, int r, int p,
                              float *X, int64_t ldX, StartState s, double gamma0, const int *slot_list,
                              const int *slot_start, const int *count, cudaStream_t st);

// on-the-fly replacement (Section 4.3): the archive of the l starts' results
struct OtfArchive {
  float *x;        // l x ldX final iterates
  float *U;        // l x ldU u = A x (objectives)
  double *F, *gamma, *f, *ev;
  int *iters, *status, *nnz;
};
// after an x-step: archive the stopped slots (scalars, then x), give the next starts to the first
// of them (new_slot[k], k < ctrl->n_new; slot_start updated; *next_start advanced)
cudaError_t launch_otf_retire(int r, int l, StartState s, int *slot_start, int *next_start, OtfArchive arc,
                              int *retire_slot, int *retire_start, int *new_slot, Ctrl *ctrl, const float *X,
                              int64_t ldx, int p, cudaStream_t st);
// Table 1 objective, explained variance and u = A x of the l archived starts (gamma: arc.gamma)
cudaError_t launch_otf_objectives(int form, const float *AT, int64_t ldat, int n, int p, OtfArchive arc, int l,
                                  int64_t ldx, int64_t ldu, double *partials, cudaStream_t st);
// f (Table 1) and the explained variance of `count` starts from the FP64 partial sums of |u_i|
// and u_i^2 (partials[(c * nchunks + b) * 2 + {0, 1}]) and ||x||_0, ||x||_1 of arc.x (gamma: arc.gamma)
cudaError_t launch_objective_reduce(int form, const double *partials, int nchunks, int p, OtfArchive arc, int count,
                                    int64_t ldx, cudaStream_t st);

// ---------------------------------------------------------------- sparse A (compressed rows)
// One CSR matrix on the device (rows x cols; indices ascending within a row, none repeated).
struct SpMat {
  const int64_t *ptr;
  const int *col;
  const float *val;
  int rows, cols;
};
// Work item of the SpMM: whole rows [row0, row1) (seg < 0), or the entries [nz0, nz1) of the long
// row row0 whose sums go to partial slot seg.  Items hold at most kSpItemNnz entries and
// kSpItemRows rows.
struct SpItem {
  int row0, row1, seg, pad;
  int64_t nz0, nz1;
};
struct SpLong {       // a row split into nseg segments, partial slots seg0 .. seg0 + nseg - 1
  int row, seg0, nseg, pad;
};
struct SpPlan {       // device arrays of items and long rows
  SpItem *items = nullptr;
  SpLong *longs = nullptr;
  int nitems = 0, nlong = 0, nseg = 0;
};
constexpr int kSpItemNnz = 2048;
constexpr int kSpItemRows = 32;
constexpr int kSpGroup = 8;     // starts per pass of the SpMM (one 32-byte sector of Bt)
constexpr int kSpSupportCap = 256;   // largest support the column scatter serves
// host side (sparse_host.cu): a CSR matrix in host memory
struct HostCsr {
  std::vector<int64_t> ptr;
  std::vector<int> col;
  std::vector<float> val;
  int64_t rows = 0, cols = 0;
};
// checks a CSR input (n x p, nnz entries) and builds the canonical A by rows and by columns
// (A^T by rows); returns nullptr, or what is wrong with the input
const char *sp_canonical(int64_t n, int64_t p, int64_t nnz, const int64_t *ptr, const int32_t *col,
                         const float *val, HostCsr *A, HostCsr *AT);
// the SpMM work items of a CSR matrix given its row offsets
void sp_plan(const std::vector<int64_t> &ptr, std::vector<SpItem> *items, std::vector<SpLong> *longs, int *nseg);
// Bt[j * ldb + k] = src[list[k] * ld + j] (list = identity when null), j < len, k < *count (rmax
// when count is null), and 0 for *count <= k < the next multiple of kSpGroup; rmax >= *count sizes
// the grid; gated
cudaError_t launch_pack_t(const float *src, int64_t ld, int len, const int *list, const int *count,
                          const int *gate, int rmax, float *Bt, int ldb, cudaStream_t st);
// out[list[k] * ldo + i] = sum_{e in row i of M} val_e Bt[col_e * ldb + k], i < M.rows, k < *count
// <= rmax (part: P.nseg x ldb floats of scratch); gated
cudaError_t launch_spmm(SpMat M, const SpPlan &P, const float *Bt, int ldb, const int *count, const int *gate,
                        const int *list, int rmax, float *out, int64_t ldo, float *part, int sms, cudaStream_t st);
// v = A^T y for y = +-1 (L1 variance): the listed rows of Y (FP32, +-1) packed as FP16 into Bt
// (A.cols x ldb16 halves, ldb16 a multiple of 16; exact), then the SpMM as above (part: row
// stride ldp floats)
cudaError_t launch_spmm_h(SpMat M, const SpPlan &P, const float *Y, int64_t ldy, int len, const int *list,
                          const int *count, int rmax, void *Bt, int ldb16, float *out, int64_t ldo, float *part,
                          int ldp, int sms, cudaStream_t st);
// u = A x over the support lists of the starts the gather serves (active, swept at least once),
// from A by columns (AT: CSR of A^T); gated
cudaError_t launch_spmv_support(SpMat AT, int n, const int *sup_idx, const float *sup_val, int cap, StartState s,
                                int r, float *U, int64_t ldu, const int *gate, cudaStream_t st);
// Projection deflation of a sparse A as a low-rank update A_k = A - W Z^T (k rows of W: n
// floats, ldw apart; of Z: p floats, ldz apart), with per-start coefficients coef (k doubles per
// start row) as scratch
struct LowRank {
  const float *W = nullptr, *Z = nullptr;
  int64_t ldw = 0, ldz = 0;
  int k = 0;
  double *coef = nullptr;
};
// out rows (list[b] or b, b < *count, or rmax when count is null) -= B^T (Cdot src): the
// coefficients Cdot_q^T src_c (FP64) into coef, then out_c -= sum_q coef_q B_q.  u -= W (Z^T x):
// src = X, Cdot = Z, B = W; v -= Z (W^T y): src = Y, Cdot = W, B = Z
cudaError_t launch_lowrank(const float *src, int64_t lds, int src_len, float *out, int64_t ldo, int out_len,
                           const int *list, const int *count, int rmax, const float *Cdot, int64_t ldc,
                           const float *B, int64_t ldb_, int k, double *coef, cudaStream_t st);
// the coefficients alone (coef rows list[b] or b)
cudaError_t launch_lowrank_coef(const float *src, int64_t lds, int src_len, const int *list, const int *count,
                                int rmax, const float *Cdot, int64_t ldc, int k, double *coef, cudaStream_t st);
// z = x / ||x||_2 (p floats); *bad = 1 when x = 0
cudaError_t launch_unit(const float *x, int p, float *z, int *bad, cudaStream_t st);
// u = A x of `count` rows of X in compensated FP32 pairs, into U; FP64 partial sums of |u_i| and
// u_i^2 per 256-row chunk to partials (count * ceil(n / 256) * 2 doubles).  With support lists
// (sup_idx / sup_val, row c at c * ldsup, nnz[c] entries), a start with at most kSpSupportCap
// nonzeros is summed over its support from A by columns (AT); the others by rows of A, their x
// packed into Bt (A.cols x ldb, ldb a multiple of 8) ldb starts at a time
// After deflation (L.k > 0) u is A_k x = A x - W (Z^T x), with L.coef holding Z^T x per start.
cudaError_t launch_fin_csr(SpMat A, SpMat AT, const float *X, int64_t ldx, int count, const int *nnz,
                           const int *sup_idx, const float *sup_val, int ldsup, float *Bt, int ldb, float *U,
                           int64_t ldu, double *partials, LowRank L, cudaStream_t st);

// Few starts (r <= kGemvMaxR): out[rows[c]][m] = sum_k P[m, k] Q[rows[c], k], c < *count (r when
// count is null; rows null = identity), m < M, streaming P once with the Q rows in shared memory
// (at most kGemvSmemMax bytes of them at a time: longer rows in chunks); gated
// Size limits from the grid's y dimension (at most 65535 blocks): several kernels put the starts
// on it, and the finalise puts a dense A's rows there in blocks of 256
constexpr int kMaxStarts = 65535;
constexpr int64_t kMaxDenseRows = 65535LL * 256;

constexpr int kGemvMaxR = 8;
constexpr int kGemvSmemMax = 200 * 1024;
int gemv_width(int r);
bool gemv_fits(int r, int64_t K);
cudaError_t launch_gemv(const float *P, int64_t ldp, int M, int K, const float *Q, int64_t ldq, const int *rows,
                        const int *count, int r, float *out, int64_t ldo, const int *gate, int sms, cudaStream_t st);

// C[m, j] = sum_k P[m, k] Q[j, k]  (both operands K-contiguous); with gate != nullptr the
// launch does nothing unless *gate != 0 (the dense u = A x is needed this sweep)
cudaError_t launch_gemm_nt_f32(const float *P, int64_t ldp, const float *Q, int64_t ldq,
                               float *C, int64_t ldc, int M, int N, int K, const int *gate,
                               cudaStream_t st);

// U[c, i] = sum_t val[c, t] AT[idx[c, t], i] for every active start; runs only when
// *gate != 0 (the control word chose the per-start gather)
cudaError_t launch_gemm1_sparse(const float *AT, int64_t ldat, int n, const int *sup_idx,
                                const float *sup_val, int cap, StartState s, int r, float *U,
                                int64_t ldu, const int *gate, cudaStream_t st);

// the same over the leading FP16 plane of A^T (low-precision sweeps): row j of that plane holds
// A[:, j] times at_scale[j], undone here with at_inv[j]
cudaError_t launch_gemm1_sparse_lowp(const void *AT0, int64_t ldat, const float *at_inv, int n, const int *sup_idx,
                                     const float *sup_val, int cap, StartState s, int r, float *U, int64_t ldu,
                                     const int *gate, cudaStream_t st);

// y-step (S1 / S2 of Table 3) for active starts.  Writes Y as FP32 (Y != nullptr, row c) and/or
// as tensor-core planes (Ypl != nullptr, row rank[c] when rank is given, else c; plane t at
// Ypl + t * plane_stride): 1 plane of +-kQScale for L1 variance, the 2 planes of kQScale y for
// L2 variance)
// With ysum (r * ceil(n / kYChunk) floats of scratch) and n > 2 kYChunk, a CTA per chunk of
// kYChunk entries and start (L2 variance: the chunks' sums of u_i^2 added in chunk order).
constexpr int kYChunk = 8192;
cudaError_t launch_ystep(int form, const float *U, int64_t ldu, int n, int r, float *Y,
                         void *Ypl, int64_t plane_stride, const int *rank, StartState s, float *X,
                         int64_t ldX, int p, float *ysum, cudaStream_t st);

// projection deflation A <- A (I - z z^T), z = x / ||x||_2, in place on the FP32 A (n x p, lda):
// *inv = 1 / ||x||_2 (0 when x = 0: A is then left as is), w (n doubles) = A z
cudaError_t launch_deflate(float *A, int64_t lda, int n, int p, const float *x, double *inv, double *w,
                           int sms, cudaStream_t st);

// ---------------------------------------------------------------- tcgen05 engine
// Operand format of the tensor-core contractions.  Every FP32 matrix they read is held as two
// FP16 planes of a power-of-two scaled copy: hi = fp16(s a), lo = fp16(s a - hi), so that
// hi + lo = s a to 22 significant bits (about 2^-22 relative; below 2^-17 of the scale's range
// an entry keeps an absolute error under 2^-38 of it).  The P operand (A for u = A x, A^T for
// v = A^T y, the union columns) has one scale per row, 2^(13 - floor(log2 max_k |a_mk|)), so
// rows of any magnitude keep their precision.  The Q operand y (|y_i| <= 1 by construction) has
// the fixed scale kQScale; x (any magnitude through spca_products) one scale per row, like P.
// The epilogue multiplies by the inverse scales, powers of two.
constexpr int kPlanes = 2;
constexpr int TC_BM_ROWS = 128;   // rows of a P tile per CTA (the contraction's M tile)
constexpr float kQScale = 16384.0f;
constexpr float kQInv = 1.0f / 16384.0f;
// per-row scales of an FP32 matrix: scale[r] = 2^(13 - floor(log2 max |src[row_map[r], :]|)) (1
// for a zero row), inv[r] = 1 / scale[r], r < rows (*rows_dev when given); gated
cudaError_t launch_row_scales(const float *src, int64_t rows, int64_t cols, int64_t lds, float *scale, float *inv,
                              const int *gate, const int *rows_dev, const int *row_map, cudaStream_t st);
struct TcPairs {      // plane products P plane a[q] x Q plane b[q], q < n; the hi x hi product
  int n;              // (a = b = 0, index first_main) accumulates apart from the corrections
  int first_main;     // (first of them at index first_corr, -1 if none)
  int first_corr;
  unsigned char a[8], b[8];
};
// plane products of the two contractions: hi x hi into the main accumulator, then the two
// correction products hi x lo and lo x hi (two general operands), or lo x (+-1) when y = +-1 is
// a single exact plane; pairs_hi: the leading planes only (low-precision sweeps)
inline TcPairs pairs_general() {
  TcPairs q{};
  q.n = 3;
  q.a[0] = 0; q.b[0] = 0;
  q.a[1] = 1; q.b[1] = 0;
  q.a[2] = 0; q.b[2] = 1;
  q.first_main = 0;
  q.first_corr = 1;
  return q;
}
inline TcPairs pairs_sign() {
  TcPairs q{};
  q.n = 2;
  q.a[0] = 0; q.b[0] = 0;
  q.a[1] = 1; q.b[1] = 0;
  q.first_main = 0;
  q.first_corr = 1;
  return q;
}
inline TcPairs pairs_hi() {
  TcPairs t{};
  t.n = 1;
  t.first_main = 0;
  t.first_corr = -1;
  t.a[0] = 0;
  t.b[0] = 0;
  return t;
}
// 3-D TMA map over `planes` FP16 planes of rows x ld (K-contiguous), box 64 x box_rows
cudaError_t make_plane_map(CUtensorMap *map, const void *base, int64_t rows, int64_t ld, int planes,
                           int box_rows, int bk);
int tc_box_rows(int nb);   // Q-operand box height for nb planes (the tile's N)
int tc_bk(int nb);         // K-block width of the contraction with nb Q planes
// P-operand map: 128-row boxes of 64-wide K blocks (each CTA loads its own 128 rows)
struct PMaps {
  CUtensorMap m[1];
};
cudaError_t make_p_maps(PMaps *maps, const void *base, int64_t rows, int64_t ld, int planes);
// out[map(c) * ldo + m] = (row_inv[m] q_inv col_inv[c]) sum_q sum_k P_{a_q}[m, k] Q_{b_q}[c, k],
// m < M, c < N (a null row_inv / col_inv counts as 1).  N bounds the
// columns for the launch; with n_dev != nullptr the kernel uses *n_dev (<= N) instead; map =
// col_map when given, else the identity.  With gate != nullptr nothing runs unless *gate != 0;
// a timed-out wait sets *err = SPCA_E_TIMEOUT
// (K from *k_dev when k_dev != nullptr, K being then only an upper bound)
// Stream-K scratch of the CTA-pair contraction: `slots` parts of tc_sk_floats_per_slot() floats
// and 2 flags per slot (zeroed by every launch).  Without it (ws == nullptr) the single-CTA kernel
// runs.
// Every wait inside the contraction kernels gives up after wait_ns nanoseconds (SPCA_E_TIMEOUT in
// *err); the owners of split tiles wait for parts flagged wait_epoch (parts are published as 1, so
// any other value is a flag that nothing sets: the test of the bounded waits).
// piece_kb: the pair kernel accumulates the main (hi x hi) product of a tile in pieces of at most
// piece_kb K-blocks (with correction products only), each in a fresh accumulator, the pieces
// summed in FP32 registers: the tensor core's accumulation truncates, so its error grows with the
// length of one accumulation.
struct TcStreamK {
  float *ws = nullptr;
  int *flags = nullptr;
  int slots = 0;
  uint64_t wait_ns = 2000000000ull;
  int wait_epoch = 1;
  int piece_kb = 40;
};
int64_t tc_sk_floats_per_slot();
cudaError_t launch_gemm_tc(const PMaps &P, int na, const CUtensorMap &Q, int nb, int M, int N, int K,
                           const int *k_dev, TcPairs pairs, float *out, int64_t ldo, const float *row_inv,
                           const float *col_inv, float q_inv, const int *gate, const int *n_dev, const int *col_map,
                           int *err, const TcStreamK &sk, cudaStream_t st);
// threshold in |v| units for U_gamma: the largest float t with t <= sqrt(gamma), so that for
// every float v, |v| > t  <=>  v^2 > gamma
inline float u_threshold(double gamma) {
  const double r = std::sqrt(gamma);
  float t = (float)r;
  if ((double)t > r) t = std::nextafterf(t, 0.0f);
  return t;
}

// ---------------------------------------------------------------- groups of problems
// One problem of a group solve: its matrix (from its handle) and its blocks of the group's
// workspace (r starts, one vector per row), in device memory.  The per-start scalars (st) of all
// problems are consecutive: problem i's starts are global starts start0 .. start0 + r - 1.
struct GProb {
  int n, p, r, start0, form;
  int64_t ldX, ldU, ldAT;
  const float *AT32;            // A^T (p x ldAT): the support gather reads columns of A as its rows
  const __half *AT16;           // or its leading FP16 plane (a resident 16-bit handle; AT32 null)
  const float *at_inv;          // with the inverse row scales of that plane
  // the member's place in its pool (the members on one matrix that share v = A^T y): its starts
  // are V's rows vbase .. vbase + r - 1, and its active starts the Y planes' rows from *yoff on
  int vbase;
  int *yoff;
  int first;                    // its first sweep is the next one (its starts are set up then)
  // the candidate x-step's scratch of the member's starts (kXstepCand values and indices, one
  // int4 of counts per start), or null
  float *cand_val;
  int *cand_idx;
  int4 *meta;
  float *X, *V, *U;             // r x ldX, r x ldX, r x ldU
  __half *Xpl, *Ypl;            // two FP16 planes each (x row-scaled, y scaled by kQScale), packed rows
  int64_t xps, yps;             // plane strides (elements)
  float *x_scale, *x_inv;       // per packed row of Xpl
  int *sup_idx;                 // r x p support lists (index, value)
  float *sup_val;
  int *act, *rank;              // active list (r)
  Ctrl *ctrl[2];                // control word of each sweep parity
  StartState st;
  XstepArgs xa;
  const float *x0;              // starts (r x ld0, device) or null (seeded: key)
  int64_t ld0;
  uint64_t key;
  double gamma0;
};
// a pool: members on one matrix whose v = A^T y has the same plane products, listed at
// members[first .. first + nmem - 1]; one contraction over their active starts side by side
struct GPool {
  int first, nmem;
  int *count;                   // active starts of all its members (device, per sweep)
  int *colmap;                  // Y row -> V row (vbase + start) of each active start
};
// per sweep, before the y-step: the pools' Y row offsets, active counts and column maps from the
// members' active lists of that parity (one CTA per pool)
cudaError_t launch_g_pools(const GPool *pools, int npool, const GProb *P, const int *members, int parity,
                           cudaStream_t st);
// the phases of a sweep for every problem of a group, one launch each (prob[g] = the problem of
// global start g, R starts in all)
// (the start initialisation runs for the members whose first sweep is next, GProb.first)
cudaError_t launch_g_start_init(const GProb *P, const int *prob, int R, cudaStream_t st);
cudaError_t launch_g_active(const GProb *P, int np, int parity, bool only_first, cudaStream_t st);
// many small device-to-device copies in one launch
struct CopyDesc {
  const void *src;
  void *dst;
  int64_t bytes;
};
cudaError_t launch_copy_list(const CopyDesc *list, int count, cudaStream_t st);
// clear (clear != 0) the control words of one parity, or gather their active counts into out[np]
cudaError_t launch_g_ctrl(const GProb *P, int np, int parity, int clear, int *out, cudaStream_t st);
cudaError_t launch_g_xplanes(const GProb *P, const int *prob, int R, cudaStream_t st);
cudaError_t launch_g_gather(const GProb *P, const int *prob, int R, int max_n, cudaStream_t st);
cudaError_t launch_g_ystep(const GProb *P, const int *prob, int R, cudaStream_t st);
// (max_p_small: the longest v that fits in shared memory, 0 if none; any_large: some v does not;
// cand: the candidate kernels first, with the problems' scratch (GProb.cand_val ...))
cudaError_t launch_g_xstep(const GProb *P, const int *prob, int R, int max_p_small, bool any_large, bool cand,
                           int parity, int sms, cudaStream_t st);
constexpr int kXstepSmemMaxP = 200 * 1024 / 4;   // the longest v the x-step stages in shared memory
constexpr int kCandMinPGroup = 512;              // shorter v: the grouped x-step's full pass only

// Grouped contraction: one persistent launch over the tiles of many contractions (one per problem
// of a group), each described by a task in device memory, its tiles listed in tile_list (task,
// local tile: M tile = local / nt, N tile = local % nt) in the order the CTAs take them.
// pmap / qmap are device addresses of tensor maps (P: 128-row boxes over two FP16 planes; Q:
// 64-row boxes over nb planes), 64-byte aligned.  Tile shapes: (bn, stages) in {64: 2, 3, 4;
// 128: 2, 3} (grouped_config_ok).
constexpr int kGroupMaxTasks = 1024;
struct GTask {
  const CUtensorMap *pmap, *qmap;
  int M, kblocks, nmax, na, nb; // output rows, K-blocks (of 64), column bound, P and Q planes loaded
  const int *n_dev;             // active columns (device; <= nmax), or null for nmax
  const int *col_map;           // output row of column c (null = c)
  float *out;
  int64_t ldo;
  const float *row_inv, *col_inv;
  float q_inv;
  TcPairs pairs;
  int mt, nt;                   // M and N tiles (N tiles of bn)
};
// lowp: every task takes the leading planes only (one accumulator per tile; tiles up to 256 wide)
bool grouped_config_ok(int bn, int stages, bool lowp);
cudaError_t launch_gemm_grouped(const GTask *tasks, const int2 *tile_list, int total_tiles, int bn, int stages,
                                bool lowp, int sms, int *err, uint64_t wait_ns, cudaStream_t st);

// FP16 planes (hi, lo; the first nplanes) of a scaled FP32 matrix, plane t at dst + t *
// plane_stride elements: destination row r is source row row_map[r] (identity when null) times
// row_scale[r] (or `scale` when row_scale is null), r < rows (*rows_dev when given); gated
cudaError_t launch_split_planes(const float *src, int64_t rows, int64_t cols, int64_t lds, void *dst,
                                int64_t ldd, int64_t plane_stride, int nplanes, const float *row_scale,
                                float scale, const int *gate, const int *rows_dev, const int *row_map,
                                cudaStream_t st);
// FP8 E4M3 operands (the low-precision sweeps of a handle stored as SPCA_FP8_E4M3_COLSCALED):
// one plane of rows x ld bytes (ld a multiple of 16), box 128 x box_rows, 128-byte swizzle
cudaError_t make_f8_map(CUtensorMap *map, const void *base, int64_t rows, int64_t ld, int box_rows);
// the pair contraction on one FP8 plane of each operand (kind::f8f6f4), FP32 accumulation; the pair
// kernel only (M > 128 and stream-K scratch), else cudaErrorInvalidValue
cudaError_t launch_gemm_tc_f8(const PMaps &P, const CUtensorMap &Q, int M, int N, int K, const int *k_dev,
                              float *out, int64_t ldo, const float *row_inv, const float *col_inv, float q_inv,
                              const int *gate, const int *n_dev, const int *col_map, int *err, const TcStreamK &sk,
                              cudaStream_t st);
// dst row r = E4M3(src row row_map[r] x row_scale[r] x mul), saturating; rows from *rows_dev when
// given; gated
cudaError_t launch_split_f8(const float *src, int64_t rows, int64_t cols, int64_t lds, uint8_t *dst, int64_t ldd,
                            const float *row_scale, float mul, const int *gate, const int *rows_dev,
                            const int *row_map, cudaStream_t st);
// dst = src x mul (n floats); gated
cudaError_t launch_scale_copy(const float *src, int n, float mul, float *dst, const int *gate, cudaStream_t st);
// u = A x over the supports from the FP8 copy of A^T (rows scaled; at_inv undoes it)
cudaError_t launch_gemm1_sparse_f8(const uint8_t *AT8, int64_t ldat, const float *at_inv, int n, const int *sup_idx,
                                   const float *sup_val, int cap, StartState s, int r, float *U, int64_t ldu,
                                   const int *gate, cudaStream_t st);
// the FP8 scales: the FP16 planes' row scales (largest entry in [2^13, 2^14)) times 2^-6, so that
// the largest entry lies in [128, 256) below E4M3's largest finite value (448); y (|y_i| <= 1)
// takes 2^7
constexpr float kF8Mul = 1.0f / 64.0f;
constexpr float kF8QScale = 128.0f;

// union S of the active starts' supports:// union S of the active starts' supports: colpos[j] = position of column j in S (or -1),
// collist[k] = the k-th column of S (k < kcap), c->kunion = |S|; then c->use_union (S fits in
// kcap columns and no start needs the dense path) and, if set, c->use_gather = 0.
// mark: p ints of scratch
cudaError_t launch_union(const int *sup_idx, int cap, StartState s, int r, int p, int *mark, int *colpos,
                         int *collist, int kcap, Ctrl *c, cudaStream_t st);
// operands of u = A x over S when c->use_union: AS planes n x kcap (row i: a_scale[i] A[i, S],
// zero past |S| up to the next multiple of 64) from the FP32 A^T, and XS planes (row k: kQScale
// times the k-th active x at the positions of S)
cudaError_t launch_union_operands(const float *AT, int64_t ldat, const float *a_scale, int n, const int *collist,
                                  int kcap, void *AS, int64_t as_pstride, const int *sup_idx,
                                  const float *sup_val, int cap, StartState s, const int *act, int nhost,
                                  const int *colpos, void *XS, int64_t xs_pstride, const Ctrl *c,
                                  cudaStream_t st);
// ordered list of the active starts (status == ST_ACTIVE): act[k] = c and rank[c] = k for the
// k-th active start; c->active = the count, c->use_gather = !c->need_dense (the union step,
// when it runs afterwards, may take the sweep over)
cudaError_t launch_active_list(const int *status, const int *nnz, int r, int *act, int *rank, Ctrl *c,
                               cudaStream_t st);

// x-step (S3..S6), objective F, stopping rule, support lists.  The candidate path needs scratch of
// kXstepCand candidates (value, index) and one int4 per start; without it every start takes the
// full pass.
constexpr int kXstepCand = 1024;
struct XstepScratch {
  float *cand_val = nullptr;   // r * kXstepCand
  int *cand_idx = nullptr;     // r * kXstepCand
  int *meta = nullptr;         // r * 4 (16-byte aligned)
};
// small problems (n p <= kSmallAlwaysEntries, or <= kSmallMaxEntries with at least
// kSmallMinStarts starts; x, y and v in shared memory): every sweep of every start in one launch,
// a CTA per start (u = A x and v = A^T y on the CUDA cores from A, the y-step writing Y, the
// full-pass x-step); sweeps = the most sweeps a start may run
constexpr int64_t kSmallAlwaysEntries = int64_t(1) << 17;
constexpr int64_t kSmallMaxEntries = int64_t(1) << 19;
constexpr int kSmallMinStarts = 16;
bool small_sweeps_fit(int64_t n, int64_t p, int r);
cudaError_t launch_small_sweeps(XstepArgs xa, const float *A, int64_t lda, int n, int p, float *X, int64_t ldx,
                                float *U, float *Y, int64_t ldu, float *V, StartState s, int *sup_idx, float *sup_val,
                                int r, int sweeps, cudaStream_t st);
cudaError_t launch_xstep(XstepArgs a, const float *V, int64_t ldv, int r, float *X, int64_t ldx,
                         StartState s, int *sup_idx, float *sup_val, Ctrl *ctrl_next, XstepScratch scratch,
                         cudaStream_t st);

// a7: Table 1 objective in FP64 for every start; u of each start into U
// (partials: r * ceil(n / 256) * 2 doubles of scratch)
cudaError_t launch_finalise(int form, const float *AT, int64_t ldat, int n, int p, const float *X,
                            int64_t ldX, StartState s, int r, float *U, int64_t ldu,
                            const int *sup_idx, const float *sup_val, int cap, double *partials,
                            cudaStream_t st);
// the same on a 16-bit copy of A^T: FP16 rows (ldat apart) times their power-of-two inverse scale
cudaError_t launch_finalise_h(int form, const __half *AT16, const float *at_inv, int64_t ldat, int n, StartState s,
                              int r, float *U, int64_t ldu, const int *sup_idx, const float *sup_val, int cap,
                              double *partials, cudaStream_t st);
// argmax over starts (ties: lower index), then y(x) and the support of the best start
cudaError_t launch_best(int form, int use_ev, StartState s, int r, int *best, cudaStream_t st);
cudaError_t launch_best_outputs(int form, const int *best, const float *U, int64_t ldu, int n,
                                const float *X, int64_t ldX, int p, float *y_out, float *x_out,
                                int64_t *support_out, int64_t *nnz_out, cudaStream_t st);

}  // namespace spca
