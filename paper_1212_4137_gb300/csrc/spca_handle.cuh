// spca_handle.cuh -- the handle of include/spca.h (a matrix on the device in the layouts the
// kernels read, plus a solve workspace), shared by the solve driver (spca_api.cu) and the group
// driver (group.cu).
#pragma once

#include <atomic>
#include <tuple>
#include <utility>
#include <vector>

#include "spca_internal.cuh"

using spca::Ctrl;
using spca::OtfArchive;
using spca::PMaps;
using spca::SpPlan;
using spca::TcStreamK;
using spca::XstepScratch;

// one captured segment of sweeps: the plan it was captured for, the executable graph, and the
// launch counts and timing events of its kernels
struct SegGraph {
  std::vector<int> key;
  cudaGraphExec_t exec = nullptr;
  int64_t counts[SPCA_K_COUNT] = {0};
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> timings;
};

// the matrix a handle holds (its copies of A, the layouts the kernels read, the deflation state),
// shared read-only by the handles spca_clone makes; freed with the last of them
struct SharedMatrix {
  std::atomic<int> refs{1};
};

struct spca_handle {
  SharedMatrix *shared = nullptr;
  int64_t n = 0, p = 0;
  int64_t ldA = 0, ldAT = 0;  // padded leading dimensions of A (n x p) and A^T (p x n)
  cudaStream_t stream = nullptr;   // the handle's own non-blocking stream (all its work)
  cudaStream_t user = nullptr;     // the caller's stream: each call starts after its prior work
  cudaEvent_t order_ev = nullptr;
  float *A32 = nullptr, *AT32 = nullptr;   // FP32 copies
  // sparse A (spca_create_csr): by rows and by columns (A^T by rows), the SpMM work items of
  // each, the packed transposed operand of the SpMM (rows x ldb, starts fastest) and the
  // partial sums of split rows
  bool sparse = false;
  int64_t *a_ptr = nullptr, *at_ptr = nullptr;
  int *a_col = nullptr, *at_col = nullptr;
  float *a_val = nullptr, *at_val = nullptr;
  SpPlan plan_a{}, plan_at{};
  float *Bt = nullptr, *sp_part = nullptr;
  int ldb = 0;
  float *ysum = nullptr;                   // chunk sums of the y-step for long u (r x ceil(n / kYChunk))
  // projection deflation of a sparse A as the low-rank update A - W Z^T: k directions z (rows of
  // Zd, p floats, ldX apart) and w = A_{i-1} z (rows of Wd, n floats, ldU apart), room for
  // defl_cap; per-start coefficients Z^T x or W^T y (lr_rows x defl_cap doubles)
  int defl_k = 0, defl_cap = 0;
  float *Wd = nullptr, *Zd = nullptr;
  double *lr_coef = nullptr;
  int lr_rows = 0;
  XstepScratch xs{};                       // the candidate x-step's lists and counts
  bool tc_ok = false;                      // the device has tcgen05 tensor cores (sm_100+)
  // SPCA_FP16_RESIDENT: only the leading FP16 planes of A and A^T (one plane each, A32 and AT32
  // freed after create); every sweep is a low-precision sweep
  bool resident16 = false;
  int sms = 1;                             // streaming multiprocessors of the device
  void *Apl = nullptr, *ATpl = nullptr;    // tensor-core planes (kPlanes FP16 each, row-scaled)
  float *a_scale = nullptr, *a_inv = nullptr;     // row scales of A (n) and their inverses
  float *at_scale = nullptr, *at_inv = nullptr;   // row scales of A^T (p) and their inverses
  PMaps pmA{}, pmAT{};                     // P-operand maps of the planes (per cluster size)
  // FP8 E4M3 copies for the low-precision sweeps (storage SPCA_FP8_E4M3_COLSCALED): A (rows scaled)
  // and A^T (A's columns scaled), their inverse scales and P-operand maps (128-row boxes)
  bool fp8 = false;
  uint8_t *A8 = nullptr, *AT8 = nullptr;
  int64_t ldA8 = 0, ldAT8 = 0;
  float *a8_inv = nullptr, *at8_inv = nullptr;
  PMaps pmA8{}, pmAT8{};

  // per-solve workspace, grown on demand
  int r_cap = 0;
  int64_t ldX = 0, ldU = 0;
  float *X = nullptr, *V = nullptr, *U = nullptr, *Y = nullptr;
  void *Xpl = nullptr, *Ypl = nullptr;     // kPlanes FP16 planes each (tensor-core engine)
  uint8_t *X8 = nullptr, *Y8 = nullptr;    // FP8 operands of the low-precision sweeps (FP8 storage)
  int64_t ldX8 = 0, ldU8 = 0;
  float *x8_inv = nullptr;
  CUtensorMap tmX8{}, tmY8{};
  float *x_scale = nullptr, *x_inv = nullptr;   // row scales of the packed X planes
  CUtensorMap tmX2{}, tmX1{}, tmY1{}, tmY2{};   // Q-operand maps: X planes (both or the leading one),
                                                // y = +-1 or the leading plane of y, y planes
  int *sup_idx = nullptr;
  float *sup_val = nullptr;
  int *act = nullptr, *rank = nullptr;     // ordered list of the active starts and its inverse
  // union of the active supports (tensor-core engine): marks, positions, columns, and the
  // compact operands of u = A x over it (kcap columns at most)
  int kcap = 0;
  int *mark = nullptr, *colpos = nullptr, *collist = nullptr;
  void *AS = nullptr, *XS = nullptr;
  PMaps pmAS{};
  CUtensorMap tmXS2{};
  int *status = nullptr, *iters = nullptr, *nnz = nullptr;
  double *F = nullptr, *F_prev = nullptr, *gamma = nullptr, *f = nullptr, *ev = nullptr;
  float *thr = nullptr, *tprev = nullptr;
  int *xfast = nullptr;
  double *partials = nullptr;
  Ctrl *ctrl = nullptr;       // device, 2 entries
  int *best = nullptr;
  float *y_out = nullptr, *x_out = nullptr;
  int64_t *support_out = nullptr, *nnz_out = nullptr;
  int *flag = nullptr;        // device scratch flag
  int *dev_err = nullptr;     // device error word written by kernels (SPCA_E_TIMEOUT)
  // on-the-fly replacement (grown on demand): the archive of the starts' results, the slots'
  // starts, the next start, the stopped / refilled slot lists, and a device copy of host x0
  int otf_l = 0, otf_r = 0;
  OtfArchive arc{};
  double *otf_partials = nullptr;
  int *slot_start = nullptr, *next_start = nullptr, *retire_slot = nullptr, *retire_start = nullptr;
  int *new_slot = nullptr;
  float *otf_x0 = nullptr;
  float *defl_x = nullptr;    // deflation: the direction (p) ...
  double *defl_w = nullptr;   // ... and w = A z (n), then 1 / ||x||
  // stream-K scratch of the CTA-pair contraction (one part per resident pair, flags)
  TcStreamK sk;
  Ctrl *h_ctrl = nullptr;     // pinned host mirror
  int *h_flag = nullptr;      // pinned host mirror (2 ints)

  // measurement hooks: launch counts, and event pairs per kernel id while profiling is on
  unsigned prof_mask = 0u;   // bit k: kernel id k is timed
  int64_t launches[SPCA_K_COUNT] = {0};
  double ms[SPCA_K_COUNT] = {0};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[SPCA_K_COUNT];
  std::vector<cudaEvent_t> event_pool;
  // graph replay of sweep segments (the sweeps between two read-backs of the control word):
  // while a segment is captured, launch counts and timing events go to the capture's lists and
  // are charged every time the graph runs
  bool capturing = false;
  int64_t cap_counts[SPCA_K_COUNT] = {0};
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> cap_timings;
  std::vector<SegGraph> graphs;          // captured segments (see spca_solve)
  int ws_gen = 0, graph_gen = 0;          // workspace generation the graphs were captured with
  unsigned graph_prof = 0u;               // and the profiling selection

  char last_error[256] = {0};
};

