// spca_api.cu -- the C ABI of include/spca.h: the handle (device copies of A in the layouts
// the kernels read), the solve driver that runs Algorithm 2 for r starts as a sequence of
// kernels on one stream, and the step-level entry points (x-step, sweep products).
#include <algorithm>
#include <atomic>
#include <tuple>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "spca_handle.cuh"

using namespace spca;

namespace {

int fail(spca_handle *h, int code, const char *fmt, const char *detail = "") {
  if (h) snprintf(h->last_error, sizeof(h->last_error), fmt, detail);
  return code;
}

#define CK(expr)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(h, e_ == cudaErrorMemoryAllocation ? SPCA_E_NOMEM : SPCA_E_CUDA,   \
                  "CUDA error: %s", cudaGetErrorString(e_));                         \
  } while (0)

#define RC(expr)                  \
  do {                            \
    int rc_ = (expr);             \
    if (rc_ != SPCA_OK) return rc_; \
  } while (0)

cudaEvent_t get_event(spca_handle *h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// runs `launch` (which enqueues `nk` kernels of kind `kid`), counting and optionally timing it
template <typename Fn>
cudaError_t timed(spca_handle *h, int kid, int nk, Fn &&launch) {
  if (h->capturing) h->cap_counts[kid] += nk;
  else h->launches[kid] += nk;
  if (!(h->prof_mask & (1u << kid))) return launch();
  cudaEvent_t a = get_event(h), b = get_event(h);
  // under stream capture an event must be an external record node to be timed after replays
  const unsigned flags = h->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  cudaError_t e = cudaEventRecordWithFlags(a, h->stream, flags);
  if (e != cudaSuccess) return e;
  e = launch();
  if (e != cudaSuccess) return e;
  e = cudaEventRecordWithFlags(b, h->stream, flags);
  if (h->capturing) h->cap_timings.emplace_back(kid, a, b);
  else h->pending[kid].push_back({a, b});
  return e;
}


void release_graphs(spca_handle *h) {
  for (SegGraph &g : h->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto &t : g.timings) {
      h->event_pool.push_back(std::get<1>(t));
      h->event_pool.push_back(std::get<2>(t));
    }
  }
  h->graphs.clear();
}

// each call's work on the handle's stream starts after the work the caller queued before it
int enter(spca_handle *h) {
  CK(cudaEventRecord(h->order_ev, h->user));
  CK(cudaStreamWaitEvent(h->stream, h->order_ev, 0));
  return SPCA_OK;
}

cudaError_t drain_profile(spca_handle *h) {
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < SPCA_K_COUNT; ++k) {
    for (auto &pr : h->pending[k]) {
      float t = 0.0f;
      cudaEventElapsedTime(&t, pr.first, pr.second);
      h->ms[k] += t;
      h->event_pool.push_back(pr.first);
      h->event_pool.push_back(pr.second);
    }
    h->pending[k].clear();
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t dalloc(T **p, size_t count, size_t elem = sizeof(T)) {
  return cudaMalloc((void **)p, count * elem + 16);
}

void free_workspace(spca_handle *h) {
  void *ptrs[] = {h->X, h->V, h->U, h->Y, h->Xpl, h->Ypl, h->sup_idx, h->sup_val, h->act, h->rank,
                  h->status, h->iters, h->nnz, h->F, h->F_prev, h->gamma, h->f, h->ev, h->thr, h->tprev, h->xfast,
                  h->partials, h->ctrl, h->best, h->y_out, h->x_out, h->support_out, h->nnz_out,
                  h->mark, h->colpos, h->collist, h->AS, h->XS, h->x_scale, h->x_inv, h->Bt, h->sp_part, h->ysum,
                  h->xs.cand_val, h->xs.cand_idx, h->xs.meta, h->X8, h->Y8, h->x8_inv};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  h->X8 = h->Y8 = nullptr;
  h->x8_inv = nullptr;
  h->Bt = h->sp_part = h->ysum = nullptr;
  h->xs = XstepScratch{};
  h->ldb = 0;
  h->mark = h->colpos = h->collist = nullptr;
  h->AS = h->XS = nullptr;
  h->X = h->V = h->U = h->Y = nullptr;
  h->Xpl = h->Ypl = nullptr;
  h->x_scale = h->x_inv = nullptr;
  h->sup_idx = nullptr; h->sup_val = nullptr;
  h->act = h->rank = nullptr;
  h->status = h->iters = h->nnz = nullptr;
  h->F = h->F_prev = h->gamma = h->f = h->ev = nullptr;
  h->thr = h->tprev = nullptr; h->xfast = nullptr; h->partials = nullptr; h->ctrl = nullptr; h->best = nullptr;
  h->y_out = h->x_out = nullptr; h->support_out = h->nnz_out = nullptr;
  h->r_cap = 0;
}

// the union of the active supports is tried while the sum of their sizes is at most this many
// times the union capacity (overlapping supports can still fit), and only while the gather it
// replaces reads at least kUnionMinReads entries of A (below that its launches cost more)
constexpr int kUnionTry = 16;
constexpr int64_t kUnionMinReads = int64_t(1) << 22;

int ensure_workspace(spca_handle *h, int r) {
  if (r <= h->r_cap) return SPCA_OK;
  release_graphs(h);   // they hold pointers into the workspace
  ++h->ws_gen;
  free_workspace(h);
  const int64_t n = h->n, p = h->p;
  h->ldX = pad_ld(p);
  h->ldU = pad_ld(n);
  const int64_t nchunks = (n + 255) / 256;
  CK(dalloc(&h->X, (size_t)r * h->ldX));
  CK(dalloc(&h->V, (size_t)r * h->ldX));
  CK(dalloc(&h->U, (size_t)r * h->ldU));
  CK(dalloc(&h->Y, (size_t)r * h->ldU));
  CK(dalloc(&h->sup_idx, (size_t)r * p));
  CK(dalloc(&h->sup_val, (size_t)r * p));
  CK(dalloc(&h->act, r)); CK(dalloc(&h->rank, r));
  CK(dalloc(&h->status, r)); CK(dalloc(&h->iters, r)); CK(dalloc(&h->nnz, r));
  CK(dalloc(&h->F, r)); CK(dalloc(&h->F_prev, r)); CK(dalloc(&h->gamma, r));
  CK(dalloc(&h->f, r)); CK(dalloc(&h->ev, r)); CK(dalloc(&h->thr, r));
  CK(dalloc(&h->tprev, r)); CK(dalloc(&h->xfast, r));
  CK(dalloc(&h->partials, (size_t)r * nchunks * 2));
  CK(dalloc(&h->ysum, (size_t)r * ((n + kYChunk - 1) / kYChunk)));
  CK(dalloc(&h->xs.cand_val, (size_t)r * kXstepCand));
  CK(dalloc(&h->xs.cand_idx, (size_t)r * kXstepCand));
  CK(dalloc(&h->xs.meta, (size_t)r * 4));
  CK(dalloc(&h->ctrl, 2)); CK(dalloc(&h->best, 1));
  CK(dalloc(&h->y_out, (size_t)h->ldU)); CK(dalloc(&h->x_out, (size_t)h->ldX));
  CK(dalloc(&h->support_out, (size_t)p)); CK(dalloc(&h->nnz_out, 1));
  // zero pads: the contractions read the padded K range
  CK(cudaMemsetAsync(h->X, 0, (size_t)r * h->ldX * sizeof(float), h->stream));
  CK(cudaMemsetAsync(h->V, 0, (size_t)r * h->ldX * sizeof(float), h->stream));
  CK(cudaMemsetAsync(h->U, 0, (size_t)r * h->ldU * sizeof(float), h->stream));
  CK(cudaMemsetAsync(h->Y, 0, (size_t)r * h->ldU * sizeof(float), h->stream));
  if (h->tc_ok) {
    CK(dalloc(&h->Xpl, (size_t)kPlanes * r * h->ldX, 2));
    CK(dalloc(&h->x_scale, (size_t)r)); CK(dalloc(&h->x_inv, (size_t)r));
    CK(dalloc(&h->Ypl, (size_t)kPlanes * r * h->ldU, 2));
    CK(cudaMemsetAsync(h->Xpl, 0, (size_t)kPlanes * r * h->ldX * 2, h->stream));
    CK(cudaMemsetAsync(h->Ypl, 0, (size_t)kPlanes * r * h->ldU * 2, h->stream));
    CK(make_plane_map(&h->tmX2, h->Xpl, r, h->ldX, 2, tc_box_rows(2), tc_bk(2)));
    CK(make_plane_map(&h->tmX1, h->Xpl, r, h->ldX, 1, tc_box_rows(1), tc_bk(1)));
    CK(make_plane_map(&h->tmY1, h->Ypl, r, h->ldU, 1, tc_box_rows(1), tc_bk(1)));
    CK(make_plane_map(&h->tmY2, h->Ypl, r, h->ldU, 2, tc_box_rows(2), tc_bk(2)));
    h->kcap = (int)std::min<int64_t>(1024, (p + 63) / 64 * 64);
    CK(dalloc(&h->mark, (size_t)p)); CK(dalloc(&h->colpos, (size_t)p)); CK(dalloc(&h->collist, (size_t)h->kcap));
    CK(dalloc(&h->AS, (size_t)kPlanes * n * h->kcap, 2));
    CK(dalloc(&h->XS, (size_t)kPlanes * r * h->kcap, 2));
    CK(make_p_maps(&h->pmAS, h->AS, n, h->kcap, 2));
    CK(make_plane_map(&h->tmXS2, h->XS, r, h->kcap, 2, tc_box_rows(2), tc_bk(2)));
  }
  if (h->fp8 && h->tc_ok) {
    h->ldX8 = (p + 15) / 16 * 16;
    h->ldU8 = (n + 15) / 16 * 16;
    CK(dalloc(&h->X8, (size_t)r * h->ldX8));
    CK(dalloc(&h->Y8, (size_t)r * h->ldU8));
    CK(dalloc(&h->x8_inv, (size_t)r));
    CK(cudaMemsetAsync(h->X8, 0, (size_t)r * h->ldX8, h->stream));
    CK(cudaMemsetAsync(h->Y8, 0, (size_t)r * h->ldU8, h->stream));
    CK(make_f8_map(&h->tmX8, h->X8, r, h->ldX8, tc_box_rows(1)));
    CK(make_f8_map(&h->tmY8, h->Y8, r, h->ldU8, tc_box_rows(1)));
  }
  if (h->sparse) {
    h->ldb = (r + kSpGroup - 1) / kSpGroup * kSpGroup;
    const int64_t bt_rows = std::max(n, p);
    const int nseg = std::max(1, std::max(h->plan_a.nseg, h->plan_at.nseg));
    CK(dalloc(&h->Bt, (size_t)bt_rows * h->ldb));
    CK(dalloc(&h->sp_part, (size_t)nseg * h->ldb));
    CK(cudaMemsetAsync(h->Bt, 0, (size_t)bt_rows * h->ldb * sizeof(float), h->stream));
  }
  h->r_cap = r;
  return SPCA_OK;
}

void free_otf(spca_handle *h) {
  void *ptrs[] = {h->arc.x, h->arc.U, h->arc.F, h->arc.gamma, h->arc.f, h->arc.ev, h->arc.iters, h->arc.status,
                  h->arc.nnz, h->otf_partials, h->slot_start, h->next_start, h->retire_slot, h->retire_start,
                  h->new_slot, h->otf_x0};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  h->arc = OtfArchive{};
  h->otf_partials = nullptr;
  h->slot_start = h->next_start = h->retire_slot = h->retire_start = h->new_slot = nullptr;
  h->otf_x0 = nullptr;
  h->otf_l = h->otf_r = 0;
}

// the on-the-fly replacement's buffers for l starts through r slots
int ensure_otf(spca_handle *h, int l, int r) {
  if (l <= h->otf_l && r <= h->otf_r) return SPCA_OK;
  release_graphs(h);   // they hold pointers into these buffers
  ++h->ws_gen;
  free_otf(h);
  const int64_t n = h->n, p = h->p;
  CK(dalloc(&h->arc.x, (size_t)l * h->ldX));
  CK(dalloc(&h->arc.U, (size_t)l * h->ldU));
  CK(dalloc(&h->arc.F, l)); CK(dalloc(&h->arc.gamma, l)); CK(dalloc(&h->arc.f, l)); CK(dalloc(&h->arc.ev, l));
  CK(dalloc(&h->arc.iters, l)); CK(dalloc(&h->arc.status, l)); CK(dalloc(&h->arc.nnz, l));
  CK(dalloc(&h->otf_partials, (size_t)l * ((n + 255) / 256) * 2));
  CK(dalloc(&h->slot_start, r)); CK(dalloc(&h->next_start, 1));
  CK(dalloc(&h->retire_slot, r)); CK(dalloc(&h->retire_start, r)); CK(dalloc(&h->new_slot, r));
  CK(dalloc(&h->otf_x0, (size_t)l * p));
  h->otf_l = l;
  h->otf_r = r;
  return SPCA_OK;
}

StartState state_of(spca_handle *h) {
  StartState s;
  s.status = h->status; s.iters = h->iters; s.nnz = h->nnz;
  s.F = h->F; s.F_prev = h->F_prev; s.gamma = h->gamma; s.thr = h->thr;
  s.f = h->f; s.ev = h->ev;
  s.tprev = h->tprev; s.xfast = h->xfast;
  return s;
}

int check_form_params(spca_handle *h, int form, double s, double gamma, int gamma_mode, int64_t p) {
  if (form < 1 || form > 8) return fail(h, SPCA_E_INVALID, "form must be 1..8%s");
  if (!std::isfinite(s) || !std::isfinite(gamma)) return fail(h, SPCA_E_INVALID, "s and gamma must be finite%s");
  if (uses_T(form) && (s < 1.0 || s > (double)p || s != std::floor(s)))
    return fail(h, SPCA_E_INVALID, "L0 constraint: s must be an integer in [1, p]%s");
  if (uses_lam(form) && s < 1.0) return fail(h, SPCA_E_INVALID, "L1 constraint: s must be >= 1%s");
  if (is_pen(form)) {
    if (gamma_mode != SPCA_GAMMA_FIXED && gamma_mode != SPCA_GAMMA_TARGET_NNZ)
      return fail(h, SPCA_E_INVALID, "unknown gamma_mode%s");
    if (gamma_mode == SPCA_GAMMA_FIXED && gamma < 0.0) return fail(h, SPCA_E_INVALID, "gamma must be >= 0%s");
    if (gamma_mode == SPCA_GAMMA_TARGET_NNZ && (s < 1.0 || s > (double)p || s != std::floor(s)))
      return fail(h, SPCA_E_INVALID, "target mode: s must be an integer in [1, p]%s");
  }
  return SPCA_OK;
}

// AUTO: the tensor cores for contractions of at least 2^26 multiply-adds (n p r), where their
// fixed costs per sweep (plane splits, the cluster launch) are small against the FP32 pipe's
// time, and for the low-precision sweeps (which need them); the CUDA cores below that and for
// up to kGemvMaxR starts (the streaming GEMV)
constexpr int64_t kTcMinMacs = int64_t(1) << 26;
int resolve_engine(spca_handle *h, int engine, int r, bool lowp, int *out) {
  if (engine != SPCA_ENGINE_AUTO && engine != SPCA_ENGINE_SIMT && engine != SPCA_ENGINE_TC)
    return fail(h, SPCA_E_INVALID, "unknown engine%s");
  if (engine == SPCA_ENGINE_TC && h->sparse)
    return fail(h, SPCA_E_UNSUPPORTED, "a sparse A runs on the CUDA-core engine%s");
  if (engine == SPCA_ENGINE_TC && !h->tc_ok)
    return fail(h, SPCA_E_UNSUPPORTED, "tensor-core engine needs an sm_100+ device%s");
  if (h->resident16 && (!lowp || engine == SPCA_ENGINE_SIMT))
    return fail(h, SPCA_E_UNSUPPORTED, "a resident 16-bit handle runs low-precision sweeps on the tensor cores only%s");
  if (engine == SPCA_ENGINE_AUTO) {
    // few starts: the streaming GEMV on the CUDA cores reads A once per product at HBM speed,
    // where the tensor-core tiles would pad the starts to 256 columns
    const bool gemv = !h->sparse && gemv_fits(r, h->n);
    engine = h->tc_ok && (lowp || (!gemv && h->n * h->p * (int64_t)r >= kTcMinMacs)) ? SPCA_ENGINE_TC
                                                                                    : SPCA_ENGINE_SIMT;
  }
  *out = engine;
  return SPCA_OK;
}

// the low-precision sweeps of an FP8 handle run on its E4M3 copies (the pair kernel: both sides of
// A above one 128-row tile and stream-K scratch; a clone's sweeps take the FP16 leading planes)
bool f8_sweeps(const spca_handle *h) {
  return h->fp8 && h->sk.ws && h->n > TC_BM_ROWS && h->p > TC_BM_ROWS;
}

SpMat sp_rows(const spca_handle *h) { return SpMat{h->a_ptr, h->a_col, h->a_val, (int)h->n, (int)h->p}; }
SpMat sp_cols(const spca_handle *h) { return SpMat{h->at_ptr, h->at_col, h->at_val, (int)h->p, (int)h->n}; }
LowRank low_rank(const spca_handle *h) {
  LowRank L;
  L.W = h->Wd;
  L.Z = h->Zd;
  L.ldw = pad_ld(h->n);
  L.ldz = pad_ld(h->p);
  L.k = h->defl_k;
  L.coef = h->lr_coef;
  return L;
}

// room for the low-rank coefficients of `rows` starts (graphs hold the old pointer: a new
// workspace generation)
int ensure_lr_coef(spca_handle *h, int rows) {
  if (h->defl_cap == 0 || rows <= h->lr_rows) return SPCA_OK;
  release_graphs(h);
  ++h->ws_gen;
  if (h->lr_coef) cudaFree(h->lr_coef);
  h->lr_coef = nullptr;
  h->lr_rows = 0;
  CK(dalloc(&h->lr_coef, (size_t)rows * h->defl_cap));
  h->lr_rows = rows;
  return SPCA_OK;
}

// deflated sparse A: u -= W (Z^T x) for the listed rows of X (the sweep's u = A x is done)
int sweep_lowrank_u(spca_handle *h, int r, const int *count, const int *list) {
  if (!h->sparse || h->defl_k == 0) return SPCA_OK;
  const LowRank L = low_rank(h);
  CK(timed(h, SPCA_K_U_DENSE, 2, [&] {
    return launch_lowrank(h->X, h->ldX, (int)h->p, h->U, h->ldU, (int)h->n, list, count, r, L.Z, L.ldz, L.W, L.ldw,
                          L.k, L.coef, h->stream);
  }));
  return SPCA_OK;
}

// sparse A: u = A x by rows for the listed rows of X (count *count, list null = the first
// *count rows): x packed transposed, then the SpMM over A's rows (gated)
int sweep_u_rows(spca_handle *h, int r, const int *gate, const int *count, const int *list) {
  const int n = (int)h->n, p = (int)h->p;
  CK(timed(h, SPCA_K_U_DENSE, 2 + (h->plan_a.nlong > 0), [&] {
    cudaError_t e = launch_pack_t(h->X, h->ldX, p, list, count, gate, r, h->Bt, h->ldb, h->stream);
    if (e != cudaSuccess) return e;
    (void)n;
    return launch_spmm(sp_rows(h), h->plan_a, h->Bt, h->ldb, count, gate, list, r, h->U, h->ldU, h->sp_part,
                       h->sms, h->stream);
  }));
  return SPCA_OK;
}

// u = A x for every active row of h->X: dense contraction (gated: runs only if *gate != 0).  The
// tensor-core engine packs the active starts (h->act, count *nact) into consecutive plane rows.
int sweep_u_dense(spca_handle *h, int engine, int r, const int *gate, const int *nact, int nhost, bool lowp,
                  const int *list = nullptr) {
  if (!list) list = h->act;
  if (h->sparse) return sweep_u_rows(h, r, gate, nact, list);
  const int n = (int)h->n, p = (int)h->p;
  cudaStream_t st = h->stream;
  if (engine == SPCA_ENGINE_TC && lowp && f8_sweeps(h)) {
    // FP8 low-precision sweep: x in E4M3 with the planes' row scales times 2^-6
    CK(timed(h, SPCA_K_U_DENSE, 4, [&] {
      cudaError_t e = launch_row_scales(h->X, nhost, p, h->ldX, h->x_scale, h->x_inv, gate, nact, list, st);
      if (e != cudaSuccess) return e;
      e = launch_split_f8(h->X, r, p, h->ldX, h->X8, h->ldX8, h->x_scale, kF8Mul, gate, nact, list, st);
      if (e != cudaSuccess) return e;
      e = launch_scale_copy(h->x_inv, r, 1.0f / kF8Mul, h->x8_inv, gate, st);
      if (e != cudaSuccess) return e;
      return launch_gemm_tc_f8(h->pmA8, h->tmX8, n, nhost, p, nullptr, h->U, h->ldU, h->a8_inv, h->x8_inv, 1.0f,
                               gate, nact, list, h->dev_err, h->sk, st);
    }));
  } else if (engine == SPCA_ENGINE_TC) {
    CK(timed(h, SPCA_K_U_DENSE, 3, [&] {
      cudaError_t e = launch_row_scales(h->X, nhost, p, h->ldX, h->x_scale, h->x_inv, gate, nact, list, st);
      if (e != cudaSuccess) return e;
      e = launch_split_planes(h->X, r, p, h->ldX, h->Xpl, h->ldX, (int64_t)h->r_cap * h->ldX, lowp ? 1 : 2,
                              h->x_scale, 1.0f, gate, nact, list, st);
      if (e != cudaSuccess) return e;
      if (lowp)
        return launch_gemm_tc(h->pmA, 1, h->tmX1, 1, n, nhost, p, nullptr, pairs_hi(), h->U, h->ldU, h->a_inv,
                              h->x_inv, 1.0f, gate, nact, list, h->dev_err, h->sk, st);
      return launch_gemm_tc(h->pmA, 2, h->tmX2, 2, n, nhost, p, nullptr, pairs_general(), h->U, h->ldU, h->a_inv,
                            h->x_inv, 1.0f, gate, nact, list, h->dev_err, h->sk, st);
    }));
  } else if (gemv_fits(r, p)) {
    CK(timed(h, SPCA_K_U_DENSE, 1, [&] {
      return launch_gemv(h->A32, h->ldA, n, p, h->X, h->ldX, list, nact, r, h->U, h->ldU, gate, h->sms, st);
    }));
  } else {
    CK(timed(h, SPCA_K_U_DENSE, 1, [&] {
      return launch_gemm_nt_f32(h->X, h->ldX, h->A32, h->ldA, h->U, h->ldU, r, n, (int)h->ldX, gate, st);
    }));
  }
  return SPCA_OK;
}

// u = A x for every active row over the union S of the active supports, when the control word
// c chose it (|S| <= h->kcap): compact FP16 operands, then the tensor-core contraction over |S|
int sweep_u_union(spca_handle *h, StartState S, const Ctrl *c, int nhost) {
  const int n = (int)h->n, p = (int)h->p;
  CK(timed(h, SPCA_K_U_SPARSE, 3, [&] {
    cudaError_t e = launch_union_operands(h->AT32, h->ldAT, h->a_scale, n, h->collist, h->kcap, h->AS,
                                          (int64_t)n * h->kcap, h->sup_idx, h->sup_val, p, S, h->act, nhost,
                                          h->colpos, h->XS, (int64_t)h->r_cap * h->kcap, c, h->stream);
    if (e != cudaSuccess) return e;
    return launch_gemm_tc(h->pmAS, 2, h->tmXS2, 2, n, nhost, h->kcap, &c->kunion, pairs_general(), h->U, h->ldU,
                          h->a_inv, nullptr, kQInv, &c->use_union, &c->active, h->act, h->dev_err, h->sk,
                          h->stream);
  }));
  return SPCA_OK;
}

// y-step and v = A^T y for every active row (tensor-core engine: packed active rows, see above)
int sweep_y_v(spca_handle *h, int engine, int form, int r, StartState S, const int *nact, int nhost,
              bool lowp = false) {
  const int n = (int)h->n, p = (int)h->p;
  cudaStream_t st = h->stream;
  const bool tc = engine == SPCA_ENGINE_TC;
  const int64_t ypstride = (int64_t)h->r_cap * h->ldU;
  if (h->sparse) {
    // y-step, y of the active starts packed transposed, the SpMM over A's columns; y = +-1 (L1
    // variance) is packed in FP16, exactly, 16 starts to a 32-byte sector
    const bool half = is_l1_var(form);
    CK(timed(h, SPCA_K_YSTEP, half ? 1 : 2, [&] {
      cudaError_t e = launch_ystep(form, h->U, h->ldU, n, r, h->Y, nullptr, 0, nullptr, S, h->X, h->ldX, p, h->ysum,
                                   st);
      if (e != cudaSuccess || half) return e;
      return launch_pack_t(h->Y, h->ldU, n, h->act, nact, nullptr, r, h->Bt, h->ldb, st);
    }));
    if (half) {
      const int ldb16 = (h->r_cap + 15) / 16 * 16;   // fits in Bt: ldb16 halves <= 2 ldb halves
      CK(timed(h, SPCA_K_V, 2 + (h->plan_at.nlong > 0), [&] {
        return launch_spmm_h(sp_cols(h), h->plan_at, h->Y, h->ldU, n, h->act, nact, r, h->Bt, ldb16, h->V, h->ldX,
                             h->sp_part, h->ldb, h->sms, st);
      }));
    } else {
      CK(timed(h, SPCA_K_V, 1 + (h->plan_at.nlong > 0), [&] {
        return launch_spmm(sp_cols(h), h->plan_at, h->Bt, h->ldb, nact, nullptr, h->act, r, h->V, h->ldX,
                           h->sp_part, h->sms, st);
      }));
    }
    if (h->defl_k > 0) {   // deflated: v -= Z (W^T y)
      const LowRank L = low_rank(h);
      CK(timed(h, SPCA_K_V, 2, [&] {
        return launch_lowrank(h->Y, h->ldU, n, h->V, h->ldX, p, h->act, nact, r, L.W, L.ldw, L.Z, L.ldz, L.k, L.coef,
                              st);
      }));
    }
    (void)nhost;
    return SPCA_OK;
  }
  // the FP8 low-precision sweep reads y as FP32 (converted to E4M3 below); the others read the planes
  const bool f8 = tc && lowp && f8_sweeps(h);
  CK(timed(h, SPCA_K_YSTEP, 1, [&] {
    return launch_ystep(form, h->U, h->ldU, n, r, tc && !f8 ? nullptr : h->Y, tc && !f8 ? h->Ypl : nullptr,
                        ypstride, tc ? h->rank : nullptr, S, h->X, h->ldX, p, h->ysum, st);
  }));
  if (f8) {
    // FP8 low-precision sweep: y (written as FP32 by the y-step) in E4M3 at scale 2^7
    CK(timed(h, SPCA_K_V, 2, [&] {
      cudaError_t e = launch_split_f8(h->Y, r, n, h->ldU, h->Y8, h->ldU8, nullptr, kF8QScale, nullptr, nact, h->act,
                                      st);
      if (e != cudaSuccess) return e;
      return launch_gemm_tc_f8(h->pmAT8, h->tmY8, p, nhost, n, nullptr, h->V, h->ldX, h->at8_inv, nullptr,
                               1.0f / kF8QScale, nullptr, nact, h->act, h->dev_err, h->sk, st);
    }));
  } else if (tc && lowp) {
    CK(timed(h, SPCA_K_V, 1, [&] {
      return launch_gemm_tc(h->pmAT, 1, h->tmY1, 1, p, nhost, n, nullptr, pairs_hi(), h->V, h->ldX, h->at_inv,
                            nullptr, kQInv, nullptr, nact, h->act, h->dev_err, h->sk, st);
    }));
  } else if (tc) {
    const bool l1 = is_l1_var(form);
    CK(timed(h, SPCA_K_V, 1, [&] {
      return launch_gemm_tc(h->pmAT, 2, l1 ? h->tmY1 : h->tmY2, l1 ? 1 : 2, p, nhost, n, nullptr,
                            l1 ? pairs_sign() : pairs_general(), h->V, h->ldX, h->at_inv, nullptr, kQInv, nullptr,
                            nact, h->act, h->dev_err, h->sk, st);
    }));
  } else if (gemv_fits(r, n)) {
    CK(timed(h, SPCA_K_V, 1, [&] {
      return launch_gemv(h->AT32, h->ldAT, p, n, h->Y, h->ldU, h->act, nact, r, h->V, h->ldX, nullptr, h->sms, st);
    }));
  } else {
    CK(timed(h, SPCA_K_V, 1, [&] {
      return launch_gemm_nt_f32(h->Y, h->ldU, h->AT32, h->ldAT, h->V, h->ldX, r, p, (int)h->ldU, nullptr, st);
    }));
  }
  return SPCA_OK;
}

int read_dev_err(spca_handle *h) {
  CK(cudaMemcpyAsync(h->h_flag + 1, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->h_flag[1] != 0) {
    const int code = h->h_flag[1];
    h->h_flag[1] = 0;
    cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream);
    return fail(h, code, "a device-side wait timed out%s");
  }
  return SPCA_OK;
}

// Projection deflation of a sparse A: A_k = A_{k-1} (I - z z^T) = A_{k-1} - w z^T with
// w = A_{k-1} z, kept as one more row of W and Z (A itself stays as given)
int deflate_sparse(spca_handle *h, const float *x, int x_is_device) {
  RC(enter(h));
  const int64_t n = h->n, p = h->p, ldw = pad_ld(n), ldz = pad_ld(p);
  cudaStream_t st = h->stream;
  RC(ensure_workspace(h, h->r_cap > 0 ? h->r_cap : 1));   // packed operand and partial sums
  if (h->defl_k == h->defl_cap) {   // grow the rows of W and Z (and the coefficients)
    const int cap = h->defl_cap ? 2 * h->defl_cap : 4;
    float *W = nullptr, *Z = nullptr;
    CK(dalloc(&W, (size_t)cap * ldw));
    cudaError_t e = dalloc(&Z, (size_t)cap * ldz);
    if (e != cudaSuccess) {
      cudaFree(W);
      CK(e);
    }
    if (h->defl_k > 0) {
      CK(cudaMemcpyAsync(W, h->Wd, (size_t)h->defl_k * ldw * sizeof(float), cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(Z, h->Zd, (size_t)h->defl_k * ldz * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    CK(cudaStreamSynchronize(st));
    cudaFree(h->Wd);
    cudaFree(h->Zd);
    h->Wd = W;
    h->Zd = Z;
    CK(cudaMemsetAsync(h->Wd + (size_t)h->defl_k * ldw, 0, (size_t)(cap - h->defl_k) * ldw * sizeof(float), st));
    CK(cudaMemsetAsync(h->Zd + (size_t)h->defl_k * ldz, 0, (size_t)(cap - h->defl_k) * ldz * sizeof(float), st));
    h->defl_cap = cap;
    const int rows = h->lr_rows > 0 ? h->lr_rows : 1;
    h->lr_rows = 0;
    RC(ensure_lr_coef(h, rows));
    release_graphs(h);
    ++h->ws_gen;
  }
  if (!h->defl_x) {
    CK(dalloc(&h->defl_x, (size_t)p));
    CK(dalloc(&h->defl_w, (size_t)n + 1));
  }
  CK(cudaMemcpyAsync(h->defl_x, x, (size_t)p * sizeof(float),
                     x_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(h->flag, 0, sizeof(int), st));
  CK(timed(h, SPCA_K_PREP, 1, [&] { return launch_check_finite(h->defl_x, 1, p, p, h->flag, st); }));
  CK(cudaMemcpyAsync(h->h_flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (*h->h_flag) return fail(h, SPCA_E_INVALID, "x has a non-finite entry%s");
  const int k = h->defl_k;
  float *z = h->Zd + (size_t)k * ldz, *w = h->Wd + (size_t)k * ldw;
  CK(timed(h, SPCA_K_PREP, 1, [&] { return launch_unit(h->defl_x, (int)p, z, h->flag, st); }));
  CK(cudaMemcpyAsync(h->h_flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (*h->h_flag) return fail(h, SPCA_E_INVALID, "x is zero%s");
  // w = A_{k-1} z = A z - W (Z^T z), by rows in compensated FP32 pairs (the finalise's product)
  const LowRank L = low_rank(h);
  CK(timed(h, SPCA_K_PREP, 3, [&] {
    cudaError_t e = launch_lowrank_coef(z, ldz, (int)p, nullptr, nullptr, 1, L.Z, L.ldz, L.k, L.coef, st);
    if (e != cudaSuccess) return e;
    return launch_fin_csr(sp_rows(h), sp_cols(h), z, ldz, 1, nullptr, nullptr, nullptr, 0, h->Bt, h->ldb, w, ldw,
                          h->partials, L, st);
  }));
  CK(cudaStreamSynchronize(st));
  h->defl_k = k + 1;
  return SPCA_OK;
}

// A^T and the tensor-core operands (row scales, FP16 planes) from the handle's FP32 A
int build_operands(spca_handle *h) {
  const int64_t n = h->n, p = h->p;
  CK(timed(h, SPCA_K_PREP, 1,
           [&] { return launch_transpose_f32(h->A32, n, p, h->ldA, h->AT32, h->ldAT, h->stream); }));
  if (!h->tc_ok) return SPCA_OK;
  CK(timed(h, SPCA_K_PREP, 4, [&] {
    cudaError_t e = launch_row_scales(h->A32, n, p, h->ldA, h->a_scale, h->a_inv, nullptr, nullptr, nullptr,
                                      h->stream);
    if (e == cudaSuccess)
      e = launch_row_scales(h->AT32, p, n, h->ldAT, h->at_scale, h->at_inv, nullptr, nullptr, nullptr, h->stream);
    const int planes = h->resident16 ? 1 : kPlanes;
    if (e == cudaSuccess)
      e = launch_split_planes(h->A32, n, h->ldA, h->ldA, h->Apl, h->ldA, n * h->ldA, planes, h->a_scale, 1.0f,
                              nullptr, nullptr, nullptr, h->stream);
    if (e == cudaSuccess)
      e = launch_split_planes(h->AT32, p, h->ldAT, h->ldAT, h->ATpl, h->ldAT, p * h->ldAT, planes, h->at_scale,
                              1.0f, nullptr, nullptr, nullptr, h->stream);
    return e;
  }));
  if (!h->fp8) return SPCA_OK;
  // FP8 copies: the planes' row scales times 2^-6 (the largest entry of a row in [128, 256))
  CK(timed(h, SPCA_K_PREP, 4, [&] {
    cudaError_t e = launch_split_f8(h->A32, n, p, h->ldA, h->A8, h->ldA8, h->a_scale, kF8Mul, nullptr, nullptr,
                                    nullptr, h->stream);
    if (e == cudaSuccess) e = launch_scale_copy(h->a_inv, (int)n, 1.0f / kF8Mul, h->a8_inv, nullptr, h->stream);
    if (e == cudaSuccess)
      e = launch_split_f8(h->AT32, p, n, h->ldAT, h->AT8, h->ldAT8, h->at_scale, kF8Mul, nullptr, nullptr, nullptr,
                          h->stream);
    if (e == cudaSuccess) e = launch_scale_copy(h->at_inv, (int)p, 1.0f / kF8Mul, h->at8_inv, nullptr, h->stream);
    return e;
  }));
  return SPCA_OK;
}

}  // namespace

extern "C" {

const char *spca_strerror(int status) {
  switch (status) {
    case SPCA_OK: return "ok";
    case SPCA_E_INVALID: return "invalid argument";
    case SPCA_E_NOMEM: return "out of memory";
    case SPCA_E_CUDA: return "CUDA error";
    case SPCA_E_TIMEOUT: return "device-side wait timed out";
    case SPCA_E_BUSY: return "handle busy";
    case SPCA_E_UNSUPPORTED: return "not supported by the library";
    default: return "unknown status";
  }
}

const char *spca_last_error(const spca_handle *h) { return h ? h->last_error : ""; }

int spca_deflate(spca_handle *h, const float *x, int x_is_device) {
  if (!h || !x) return fail(h, SPCA_E_INVALID, "NULL argument%s");
  if (h->shared && h->shared->refs.load() > 1)
    return fail(h, SPCA_E_UNSUPPORTED, "the matrix is shared with another handle (spca_clone)%s");
  if (h->sparse) return deflate_sparse(h, x, x_is_device);
  if (h->resident16) return fail(h, SPCA_E_UNSUPPORTED, "deflation of a resident 16-bit handle%s");
  RC(enter(h));
  const int64_t n = h->n, p = h->p;
  cudaStream_t st = h->stream;
  if (!h->defl_x) {
    CK(dalloc(&h->defl_x, (size_t)p));
    CK(dalloc(&h->defl_w, (size_t)n + 1));
  }
  CK(cudaMemcpyAsync(h->defl_x, x, (size_t)p * sizeof(float),
                     x_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  // x must be finite and nonzero
  CK(cudaMemsetAsync(h->flag, 0, sizeof(int), st));
  CK(timed(h, SPCA_K_PREP, 1, [&] { return launch_check_finite(h->defl_x, 1, p, p, h->flag, st); }));
  CK(cudaMemcpyAsync(h->h_flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (*h->h_flag) return fail(h, SPCA_E_INVALID, "x has a non-finite entry%s");
  CK(timed(h, SPCA_K_PREP, 3, [&] {
    return launch_deflate(h->A32, h->ldA, (int)n, (int)p, h->defl_x, h->defl_w + n, h->defl_w, h->sms, st);
  }));
  double inv = 0.0;
  CK(cudaMemcpyAsync(&inv, h->defl_w + n, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (!(inv > 0.0)) return fail(h, SPCA_E_INVALID, "x is zero%s");
  RC(build_operands(h));
  CK(cudaStreamSynchronize(st));
  return SPCA_OK;
}

int spca_set_waits(spca_handle *h, int64_t wait_limit_us, int unpublished_parts) {
  if (!h) return SPCA_E_INVALID;
  if (wait_limit_us < 1 || wait_limit_us > 60000000) return fail(h, SPCA_E_INVALID, "wait_limit_us out of range%s");
  CK(cudaStreamSynchronize(h->stream));
  release_graphs(h);   // captured launches hold the old settings
  ++h->ws_gen;
  h->sk.wait_ns = (uint64_t)wait_limit_us * 1000ull;
  h->sk.wait_epoch = unpublished_parts ? 2 : 1;   // parts are published as 1
  return SPCA_OK;
}

int spca_profile_enable(spca_handle *h, int mask) {
  if (!h || mask < 0 || mask > SPCA_PROFILE_ALL) return SPCA_E_INVALID;
  CK(drain_profile(h));
  for (int k = 0; k < SPCA_K_COUNT; ++k) {
    h->launches[k] = 0;
    h->ms[k] = 0.0;
  }
  h->prof_mask = (unsigned)mask;
  return SPCA_OK;
}

int spca_profile_query(spca_handle *h, int kernel, int64_t *launches, double *ms) {
  if (!h || kernel < SPCA_K_ALL || kernel >= SPCA_K_COUNT) return SPCA_E_INVALID;
  CK(drain_profile(h));
  int64_t l = 0;
  double t = 0.0;
  for (int k = 0; k < SPCA_K_COUNT; ++k) {
    if (kernel == SPCA_K_ALL || kernel == k) {
      l += h->launches[k];
      t += h->ms[k];
    }
  }
  if (launches) *launches = l;
  if (ms) *ms = t;
  return SPCA_OK;
}

void spca_destroy(spca_handle *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  release_graphs(h);
  drain_profile(h);
  for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
  free_workspace(h);
  free_otf(h);
  // this handle's own buffers
  void *own[] = {h->flag, h->dev_err, h->sk.ws, h->sk.flags, h->defl_x, h->defl_w, h->lr_coef};
  for (void *q : own)
    if (q) cudaFree(q);
  // the matrix, with the last handle that holds it
  if (!h->shared || h->shared->refs.fetch_sub(1) == 1) {
    void *mat[] = {h->A32, h->AT32, h->Apl, h->ATpl, h->a_scale, h->a_inv, h->at_scale, h->at_inv, h->A8, h->AT8,
                   h->a8_inv, h->at8_inv,
                   h->a_ptr, h->a_col, h->a_val, h->at_ptr, h->at_col, h->at_val, h->Wd, h->Zd,
                   h->plan_a.items, h->plan_a.longs, h->plan_at.items, h->plan_at.longs};
    for (void *q : mat)
      if (q) cudaFree(q);
    delete h->shared;
  }
  if (h->h_ctrl) cudaFreeHost(h->h_ctrl);
  if (h->h_flag) cudaFreeHost(h->h_flag);
  if (h->order_ev) cudaEventDestroy(h->order_ev);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int spca_create(spca_handle **out, const void *A, int64_t n, int64_t p, int64_t lda, int in_dtype,
                int a_is_device, int storage, void *cuda_stream) {
  spca_handle *h = nullptr;
  if (!out || !A) return SPCA_E_INVALID;
  if (n < 1 || p < 1 || lda < p || n > INT32_MAX || p > INT32_MAX) return SPCA_E_INVALID;
  if (n > kMaxDenseRows) return SPCA_E_UNSUPPORTED;
  if (in_dtype != SPCA_F32 && in_dtype != SPCA_F64) return SPCA_E_INVALID;
  if (storage != SPCA_F32 && storage != SPCA_FP16 && storage != SPCA_FP8_E4M3_COLSCALED &&
      storage != SPCA_FP16_RESIDENT) {
    if (storage == SPCA_F64) return SPCA_E_UNSUPPORTED;
    return SPCA_E_INVALID;
  }
  int ndev = 0, dev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SPCA_E_CUDA;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPCA_E_CUDA;
  h = new (std::nothrow) spca_handle();
  if (!h) return SPCA_E_NOMEM;
  h->shared = new (std::nothrow) SharedMatrix();
  if (!h->shared) {
    delete h;
    return SPCA_E_NOMEM;
  }
  int rc = [&]() -> int {
    h->n = n; h->p = p;
    h->user = (cudaStream_t)cuda_stream;
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->order_ev, cudaEventDisableTiming));
    RC(enter(h));
    h->ldA = pad_ld(p);
    h->ldAT = pad_ld(n);
    int major = 0;
    CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    h->tc_ok = major >= 10;
    CK(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev));
    if ((storage == SPCA_FP16 || storage == SPCA_FP8_E4M3_COLSCALED || storage == SPCA_FP16_RESIDENT) && !h->tc_ok)
      return SPCA_E_UNSUPPORTED;   // the planes need tcgen05
    h->fp8 = storage == SPCA_FP8_E4M3_COLSCALED;
    h->resident16 = storage == SPCA_FP16_RESIDENT;
    const int planes = h->resident16 ? 1 : kPlanes;
    CK(cudaMallocHost((void **)&h->h_ctrl, 2 * sizeof(Ctrl)));
    CK(cudaMallocHost((void **)&h->h_flag, 2 * sizeof(int)));
    h->h_flag[0] = h->h_flag[1] = 0;
    CK(dalloc(&h->flag, 1));
    CK(dalloc(&h->dev_err, 1));
    CK(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream));
    CK(dalloc(&h->A32, (size_t)n * h->ldA));
    CK(dalloc(&h->AT32, (size_t)p * h->ldAT));
    CK(cudaMemsetAsync(h->A32, 0, (size_t)n * h->ldA * sizeof(float), h->stream));
    CK(cudaMemsetAsync(h->AT32, 0, (size_t)p * h->ldAT * sizeof(float), h->stream));
    const cudaMemcpyKind kind = a_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (in_dtype == SPCA_F32) {
      CK(cudaMemcpy2DAsync(h->A32, h->ldA * sizeof(float), A, lda * sizeof(float), p * sizeof(float), n, kind,
                           h->stream));
    } else {
      double *tmp = nullptr;
      CK(dalloc(&tmp, (size_t)n * lda));
      cudaError_t e = cudaMemcpyAsync(tmp, A, (size_t)n * lda * sizeof(double), kind, h->stream);
      if (e == cudaSuccess) e = launch_convert_f64_f32(tmp, n, p, lda, h->A32, h->ldA, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      cudaFree(tmp);
      CK(e);
    }
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    CK(timed(h, SPCA_K_PREP, 1, [&] { return launch_check_finite(h->A32, n, p, h->ldA, h->flag, h->stream); }));
    CK(cudaMemcpyAsync(h->h_flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    if (h->tc_ok) {
      CK(dalloc(&h->Apl, (size_t)planes * n * h->ldA, 2));
      CK(dalloc(&h->ATpl, (size_t)planes * p * h->ldAT, 2));
      CK(dalloc(&h->a_scale, (size_t)n)); CK(dalloc(&h->a_inv, (size_t)n));
      CK(dalloc(&h->at_scale, (size_t)p)); CK(dalloc(&h->at_inv, (size_t)p));
    }
    if (h->fp8) {
      h->ldA8 = (p + 15) / 16 * 16;
      h->ldAT8 = (n + 15) / 16 * 16;
      CK(dalloc(&h->A8, (size_t)n * h->ldA8));
      CK(dalloc(&h->AT8, (size_t)p * h->ldAT8));
      CK(cudaMemsetAsync(h->A8, 0, (size_t)n * h->ldA8, h->stream));
      CK(cudaMemsetAsync(h->AT8, 0, (size_t)p * h->ldAT8, h->stream));
      CK(dalloc(&h->a8_inv, (size_t)n)); CK(dalloc(&h->at8_inv, (size_t)p));
      CK(make_f8_map(&h->pmA8.m[0], h->A8, n, h->ldA8, TC_BM_ROWS));
      CK(make_f8_map(&h->pmAT8.m[0], h->AT8, p, h->ldAT8, TC_BM_ROWS));
    }
    RC(build_operands(h));
    if (h->tc_ok) {
      CK(make_p_maps(&h->pmA, h->Apl, n, h->ldA, planes));
      CK(make_p_maps(&h->pmAT, h->ATpl, p, h->ldAT, planes));
      h->sk.slots = h->sms / 2 > 0 ? h->sms / 2 : 1;
      CK(dalloc(&h->sk.ws, (size_t)h->sk.slots * tc_sk_floats_per_slot()));
      CK(dalloc(&h->sk.flags, (size_t)2 * h->sk.slots));
      CK(cudaMemsetAsync(h->sk.flags, 0, (size_t)2 * h->sk.slots * sizeof(int), h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    if (*h->h_flag) return fail(h, SPCA_E_INVALID, "A has a non-finite entry%s");
    if (h->resident16) {   // the planes are built: the FP32 copies go
      CK(cudaFree(h->A32));
      h->A32 = nullptr;
      CK(cudaFree(h->AT32));
      h->AT32 = nullptr;
    }
    return SPCA_OK;
  }();
  if (rc != SPCA_OK) {
    spca_destroy(h);
    return rc;
  }
  *out = h;
  return SPCA_OK;
}

int spca_create_csr(spca_handle **out, int64_t n, int64_t p, int64_t nnz, const int64_t *row_ptr,
                    const int32_t *col_idx, const float *values, int is_device, void *cuda_stream) {
  spca_handle *h = nullptr;
  if (!out || !row_ptr || (nnz > 0 && (!col_idx || !values))) return SPCA_E_INVALID;
  if (n < 1 || p < 1 || nnz < 0 || n > INT32_MAX || p > INT32_MAX || nnz > INT32_MAX) return SPCA_E_INVALID;
  int ndev = 0, dev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SPCA_E_CUDA;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPCA_E_CUDA;
  h = new (std::nothrow) spca_handle();
  if (!h) return SPCA_E_NOMEM;
  h->shared = new (std::nothrow) SharedMatrix();
  if (!h->shared) {
    delete h;
    return SPCA_E_NOMEM;
  }
  int rc = [&]() -> int {
    h->n = n; h->p = p;
    h->sparse = true;
    h->tc_ok = false;   // the sweeps run on the sparse CUDA-core kernels
    h->user = (cudaStream_t)cuda_stream;
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->order_ev, cudaEventDisableTiming));
    RC(enter(h));
    CK(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaMallocHost((void **)&h->h_ctrl, 2 * sizeof(Ctrl)));
    CK(cudaMallocHost((void **)&h->h_flag, 2 * sizeof(int)));
    h->h_flag[0] = h->h_flag[1] = 0;
    CK(dalloc(&h->flag, 1));
    CK(dalloc(&h->dev_err, 1));
    CK(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream));
    // the input on the host (the canonical layouts are built there)
    std::vector<int64_t> hp;
    std::vector<int32_t> hc;
    std::vector<float> hv;
    const int64_t *P = row_ptr;
    const int32_t *Cc = col_idx;
    const float *Vv = values;
    if (is_device) {
      hp.resize((size_t)n + 1);
      hc.resize((size_t)nnz);
      hv.resize((size_t)nnz);
      CK(cudaMemcpyAsync(hp.data(), row_ptr, hp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
      if (nnz > 0) {
        CK(cudaMemcpyAsync(hc.data(), col_idx, hc.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(hv.data(), values, hv.size() * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
      }
      CK(cudaStreamSynchronize(h->stream));
      P = hp.data();
      Cc = hc.data();
      Vv = hv.data();
    }
    HostCsr A, AT;
    if (const char *bad = sp_canonical(n, p, nnz, P, Cc, Vv, &A, &AT)) return fail(h, SPCA_E_INVALID, "%s", bad);
    const size_t m = A.col.size();
    CK(dalloc(&h->a_ptr, (size_t)n + 1));
    CK(dalloc(&h->at_ptr, (size_t)p + 1));
    CK(dalloc(&h->a_col, m + 1)); CK(dalloc(&h->a_val, m + 1));
    CK(dalloc(&h->at_col, m + 1)); CK(dalloc(&h->at_val, m + 1));
    CK(cudaMemcpyAsync(h->a_ptr, A.ptr.data(), A.ptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->at_ptr, AT.ptr.data(), AT.ptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                       h->stream));
    if (m > 0) {
      CK(cudaMemcpyAsync(h->a_col, A.col.data(), m * sizeof(int), cudaMemcpyHostToDevice, h->stream));
      CK(cudaMemcpyAsync(h->a_val, A.val.data(), m * sizeof(float), cudaMemcpyHostToDevice, h->stream));
      CK(cudaMemcpyAsync(h->at_col, AT.col.data(), m * sizeof(int), cudaMemcpyHostToDevice, h->stream));
      CK(cudaMemcpyAsync(h->at_val, AT.val.data(), m * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    }
    // the SpMM work items of both layouts
    for (int side = 0; side < 2; ++side) {
      std::vector<SpItem> items;
      std::vector<SpLong> longs;
      SpPlan &pl = side == 0 ? h->plan_a : h->plan_at;
      sp_plan(side == 0 ? A.ptr : AT.ptr, &items, &longs, &pl.nseg);
      pl.nitems = (int)items.size();
      pl.nlong = (int)longs.size();
      CK(dalloc(&pl.items, items.size() + 1));
      CK(dalloc(&pl.longs, longs.size() + 1));
      if (!items.empty())
        CK(cudaMemcpyAsync(pl.items, items.data(), items.size() * sizeof(SpItem), cudaMemcpyHostToDevice, h->stream));
      if (!longs.empty())
        CK(cudaMemcpyAsync(pl.longs, longs.data(), longs.size() * sizeof(SpLong), cudaMemcpyHostToDevice,
                           h->stream));
      CK(cudaStreamSynchronize(h->stream));   // the host vectors go out of scope
    }
    return SPCA_OK;
  }();
  if (rc != SPCA_OK) {
    spca_destroy(h);
    return rc;
  }
  *out = h;
  return SPCA_OK;
}

int spca_clone(spca_handle **out, spca_handle *src, void *cuda_stream) {
  if (!out || !src || !src->shared) return SPCA_E_INVALID;
  spca_handle *h = new (std::nothrow) spca_handle();
  if (!h) return SPCA_E_NOMEM;
  // the matrix: shared, read-only
  h->shared = src->shared;
  h->shared->refs.fetch_add(1);
  h->n = src->n; h->p = src->p;
  h->ldA = src->ldA; h->ldAT = src->ldAT;
  h->A32 = src->A32; h->AT32 = src->AT32;
  h->sparse = src->sparse;
  h->a_ptr = src->a_ptr; h->at_ptr = src->at_ptr;
  h->a_col = src->a_col; h->at_col = src->at_col;
  h->a_val = src->a_val; h->at_val = src->at_val;
  h->plan_a = src->plan_a; h->plan_at = src->plan_at;
  h->defl_k = src->defl_k; h->defl_cap = src->defl_cap;
  h->Wd = src->Wd; h->Zd = src->Zd;
  h->tc_ok = src->tc_ok; h->sms = src->sms;
  h->resident16 = src->resident16;
  h->Apl = src->Apl; h->ATpl = src->ATpl;
  h->a_scale = src->a_scale; h->a_inv = src->a_inv;
  h->at_scale = src->at_scale; h->at_inv = src->at_inv;
  h->pmA = src->pmA; h->pmAT = src->pmAT;
  h->fp8 = src->fp8;
  h->A8 = src->A8; h->AT8 = src->AT8;
  h->ldA8 = src->ldA8; h->ldAT8 = src->ldAT8;
  h->a8_inv = src->a8_inv; h->at8_inv = src->at8_inv;
  h->pmA8 = src->pmA8; h->pmAT8 = src->pmAT8;
  int rc = [&]() -> int {
    h->user = (cudaStream_t)cuda_stream;
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->order_ev, cudaEventDisableTiming));
    RC(enter(h));
    CK(cudaMallocHost((void **)&h->h_ctrl, 2 * sizeof(Ctrl)));
    CK(cudaMallocHost((void **)&h->h_flag, 2 * sizeof(int)));
    h->h_flag[0] = h->h_flag[1] = 0;
    CK(dalloc(&h->flag, 1));
    CK(dalloc(&h->dev_err, 1));
    CK(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream));
    // no stream-K scratch: its schedule needs every CTA of a launch resident at once, which
    // launches of other handles running at the same time cannot guarantee; the contractions take
    // the cluster kernel, whose CTAs never wait for other clusters
    CK(cudaStreamSynchronize(h->stream));
    return SPCA_OK;
  }();
  if (rc != SPCA_OK) {
    spca_destroy(h);
    return rc;
  }
  *out = h;
  return SPCA_OK;
}

int spca_xstep(spca_handle *h, int form, double s, double gamma, int calibrate, const float *V, int64_t ldv,
               int r, float *X, int64_t ldx, double *F, int *nnz, double *thr) {
  if (!h || !V || !X || !F || !nnz || !thr || r < 1) return fail(h, SPCA_E_INVALID, "bad argument%s");
  if (ldv < h->p || ldx < h->p) return fail(h, SPCA_E_INVALID, "leading dimension < p%s");
  RC(check_form_params(h, form, s, gamma, calibrate ? SPCA_GAMMA_TARGET_NNZ : SPCA_GAMMA_FIXED, h->p));
  XstepArgs a{};
  a.form = form; a.p = (int)h->p; a.s = s;
  a.calibrate = is_pen(form) && calibrate;
  a.per_start_thr = 0;
  a.thr_fixed = uses_U(form) ? u_threshold(gamma) : (float)gamma;
  a.gamma_fixed = gamma;
  a.stop_test = 0; a.tol = -1.0; a.max_iter = 1 << 30;
  a.cap = 0; a.sparse_cap = (int)h->p;
  StartState st{};
  st.nnz = nnz; st.F = F; st.gamma = thr;
  RC(enter(h));
  CK(timed(h, SPCA_K_XSTEP, 1, [&] {
    return launch_xstep(a, V, ldv, r, X, ldx, st, nullptr, nullptr, nullptr, XstepScratch{}, h->stream);
  }));
  CK(cudaStreamSynchronize(h->stream));
  return SPCA_OK;
}

int spca_products(spca_handle *h, int form, int engine, const float *X, int64_t ldx, int r, float *U,
                  int64_t ldu, float *V, int64_t ldv) {
  if (!h || !X || !U || !V || r < 1) return fail(h, SPCA_E_INVALID, "bad argument%s");
  if (r > kMaxStarts) return fail(h, SPCA_E_UNSUPPORTED, "more than 65535 rows%s");
  if (form < 1 || form > 8) return fail(h, SPCA_E_INVALID, "form must be 1..8%s");
  if (ldx < h->p || ldv < h->p || ldu < h->n) return fail(h, SPCA_E_INVALID, "leading dimension too small%s");
  const bool lowp = engine == SPCA_ENGINE_TC_LOWP;
  int eng;
  RC(resolve_engine(h, lowp ? SPCA_ENGINE_TC : engine, r, lowp, &eng));
  RC(enter(h));
  RC(ensure_workspace(h, r));
  RC(ensure_lr_coef(h, r));
  const int n = (int)h->n, p = (int)h->p;
  cudaStream_t st = h->stream;
  CK(cudaMemcpy2DAsync(h->X, h->ldX * sizeof(float), X, ldx * sizeof(float), (size_t)p * sizeof(float), r,
                       cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(h->status, 0xFF, (size_t)r * sizeof(int), st));   // every row active (-1)
  CK(cudaMemsetAsync(h->iters, 0, (size_t)r * sizeof(int), st));
  CK(cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), st));
  CK(launch_active_list(h->status, nullptr, r, h->act, h->rank, &h->ctrl[0], st));
  RC(sweep_u_dense(h, eng, r, nullptr, &h->ctrl[0].active, r, lowp));
  RC(sweep_lowrank_u(h, r, &h->ctrl[0].active, h->act));
  RC(sweep_y_v(h, eng, form, r, state_of(h), &h->ctrl[0].active, r, lowp));
  CK(cudaMemcpy2DAsync(U, ldu * sizeof(float), h->U, h->ldU * sizeof(float), (size_t)n * sizeof(float), r,
                       cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpy2DAsync(V, ldv * sizeof(float), h->V, h->ldX * sizeof(float), (size_t)p * sizeof(float), r,
                       cudaMemcpyDeviceToDevice, st));
  RC(read_dev_err(h));
  return SPCA_OK;
}

int spca_solve(spca_handle *h, const spca_params *prm, const float *x0, spca_result *res) {
  if (!h || !prm || !res) return fail(h, SPCA_E_INVALID, "NULL argument%s");
  const spca_params P = *prm;
  const int form = P.form;
  RC(check_form_params(h, form, P.s, P.gamma, P.gamma_mode, h->p));
  if (P.r < 1 || P.max_iter < 1) return fail(h, SPCA_E_INVALID, "r and max_iter must be >= 1%s");
  if (!std::isfinite(P.tol)) return fail(h, SPCA_E_INVALID, "tol must be finite%s");
  const bool target = is_pen(form) && P.gamma_mode == SPCA_GAMMA_TARGET_NNZ;
  if (target && P.gamma_calib_sweeps < 1) return fail(h, SPCA_E_INVALID, "gamma_calib_sweeps must be >= 1%s");
  if (P.lowp_sweeps < 0 || P.refine_sweeps < 0 || P.timeout_us < 0 || P.lowp_first < 0)
    return fail(h, SPCA_E_INVALID, "lowp_sweeps, lowp_first, refine_sweeps and timeout_us must be >= 0%s");
  // a resident 16-bit handle: every sweep reads the 16-bit copy (no FP32 copy to refine on)
  const bool all_lowp = h->resident16;
  if (all_lowp && (P.lowp_sweeps > 0 || P.lowp_first > 0 || P.refine_sweeps > 0))
    return fail(h, SPCA_E_INVALID,
                "every sweep of a resident 16-bit handle is a low-precision sweep: lowp_sweeps, lowp_first and "
                "refine_sweeps must be 0%s");
  int engine;
  RC(resolve_engine(h, P.engine, P.r, P.lowp_sweeps > 0 || all_lowp, &engine));
  if (P.lowp_sweeps > 0 && engine != SPCA_ENGINE_TC)
    return fail(h, SPCA_E_UNSUPPORTED, "low-precision sweeps need the tensor-core engine%s");
  // on-the-fly replacement: l starts through the r slots
  const int l = P.total_starts > P.r ? P.total_starts : P.r;
  if (l > kMaxStarts) return fail(h, SPCA_E_UNSUPPORTED, "more than 65535 starts%s");
  const bool otf = l > P.r;
  if (otf && (P.lowp_sweeps > 0 || all_lowp))
    return fail(h, SPCA_E_UNSUPPORTED, "low-precision sweeps with on-the-fly replacement%s");
  RC(enter(h));
  const auto t_start = std::chrono::steady_clock::now();
  // low-precision sweeps: F0 FP32 sweeps first, then L low-precision ones, then FP32 again (all
  // of them for a resident 16-bit handle)
  const int L = all_lowp ? P.max_iter : P.lowp_sweeps, F0 = P.lowp_sweeps > 0 ? P.lowp_first : 0;
  const int max_iter = P.refine_sweeps > 0 ? (int)std::min<int64_t>(P.max_iter, (int64_t)F0 + L + P.refine_sweeps)
                                           : P.max_iter;

  const int r = P.r, n = (int)h->n, p = (int)h->p;
  RC(ensure_workspace(h, r));
  if (otf) RC(ensure_otf(h, l, r));
  RC(ensure_lr_coef(h, l));
  cudaStream_t st = h->stream;
  StartState S = state_of(h);

  // ---- a1: starting points
  const double gamma0 = is_pen(form) && !target ? P.gamma : 0.0;
  // the starts' source: x0 rows (copied into X for a plain solve, kept whole for on-the-fly
  // replacement, where slots take later rows), or the seeded stream
  const float *x0src = nullptr;
  int64_t ld0 = 0;
  if (x0) {
    if (otf) {
      if (P.x0_is_device) {
        x0src = x0;
      } else {
        CK(cudaMemcpyAsync(h->otf_x0, x0, (size_t)l * p * sizeof(float), cudaMemcpyHostToDevice, st));
        x0src = h->otf_x0;
      }
      ld0 = p;
    } else {
      CK(cudaMemcpy2DAsync(h->X, h->ldX * sizeof(float), x0, (size_t)p * sizeof(float), (size_t)p * sizeof(float),
                           r, P.x0_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
      x0src = h->X;
      ld0 = h->ldX;
    }
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), st));
    CK(timed(h, SPCA_K_PREP, 1,
             [&] { return launch_check_finite(x0src, otf ? l : r, p, ld0, h->flag, st); }));
    CK(cudaMemcpyAsync(h->h_flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (*h->h_flag) return fail(h, SPCA_E_INVALID, "x0 has a non-finite entry%s");
  }
  CK(timed(h, SPCA_K_INIT, 1, [&] {
    return launch_start_init(x0src, ld0, P.seed, r, p, h->X, h->ldX, S, gamma0, nullptr, nullptr, nullptr, st);
  }));
  std::vector<int> iota;
  if (otf) {   // slot c holds start c; the next start is r
    iota.resize(r + 1);
    for (int c = 0; c < r; ++c) iota[c] = c;
    iota[r] = r;
    CK(cudaMemcpyAsync(h->slot_start, iota.data(), r * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->next_start, iota.data() + r, sizeof(int), cudaMemcpyHostToDevice, st));
  }
  memset(&h->h_ctrl[0], 0, sizeof(Ctrl));
  h->h_ctrl[0].active = r;
  h->h_ctrl[0].need_dense = 1;      // x^(0) is dense: the first sweep's u = A x is the dense one
  CK(cudaMemcpyAsync(h->ctrl, h->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  CK(timed(h, SPCA_K_XSTEP, 1,
           [&] { return launch_active_list(h->status, nullptr, r, h->act, h->rank, &h->ctrl[0], st); }));
  CK(cudaMemcpyAsync(h->h_ctrl + 1, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));  // h_ctrl is reused below
  int nhost = h->h_ctrl[1].active;  // active starts as the host knows them (sizes the launches)

  // ---- the sweeps (Algorithm 2)
  XstepArgs xa{};
  xa.form = form; xa.p = p; xa.s = P.s;
  xa.thr_fixed = uses_U(form) ? u_threshold(P.gamma) : (float)P.gamma;
  xa.gamma_fixed = P.gamma;
  xa.tol = P.tol; xa.max_iter = max_iter;
  xa.cap = p;
  // the support gather takes supports up to sparse_cap; a sparse A's gather scatters the
  // support's columns one at a time, so it pays only for small supports
  xa.sparse_cap = h->sparse ? std::min(p, kSpSupportCap) : (p / 8 > 0 ? p / 8 : 1);
  const int C = target ? P.gamma_calib_sweeps : 0;
  // the x-step's switches follow each start's own sweep count (calibration sweeps of Section 4.1,
  // then the frozen gamma; the stopping rule compares two FP32 sweeps)
  xa.schedule = 1;
  xa.target = target ? 1 : 0;
  xa.calib_sweeps = C;
  // the stopping rule compares FP32 sweeps after the window (any two sweeps when all are
  // low-precision ones)
  xa.lowp_sweeps = all_lowp ? 0 : F0 + L;
  xa.stop_enabled = P.tol >= 0.0 ? 1 : 0;
  // the host queues this many sweeps before it reads the active count back; every path decision
  // inside a sweep is taken on the device from the control word
  const int check_every = 4;
  // the union of the active supports is built only while the sum of their sizes (read back
  // with the active count; dense before the first read) could let it fit the union operands
  int64_t sum_nnz = (int64_t)nhost * p;
  bool union_built = false;
  // the dense u = A x is a faster path for large supports, never a required one (the gather
  // takes any support): the host queues it only while some active support may come near
  // sparse_cap (T_s keeps at most s entries; otherwise read back with the active count), and the
  // x-step of the sweep before requests it only then
  const int sparse_cap = xa.sparse_cap;
  int64_t max_nnz = uses_T(form) ? std::min<int64_t>((int64_t)P.s, p) : p;
  bool dense_queued = true;   // x^(0) is dense
  // The sweeps are queued in segments that end at a read-back (every check_every sweeps).  A
  // segment's host decisions (the plan: which optional launches, the x-step's switches) are made
  // up front from the last read-back; its kernels are captured into a CUDA graph once per distinct
  // plan and replayed, so that in steady state a segment is one launch.
  struct SweepPlan {
    int k;
    bool lowp, dense_in, union_in, union_out;
    int sparse_cap;
  };
  auto enqueue = [&](const SweepPlan &pl) -> int {
    Ctrl *cur = h->ctrl + ((pl.k - 1) & 1), *nxt = h->ctrl + (pl.k & 1);
    // u = A x: over the union of the supports when it is small (tensor cores), else the dense
    // contraction, or the per-start support gather when every support is small
    if (pl.dense_in) RC(sweep_u_dense(h, engine, r, &cur->need_dense, &cur->active, r, pl.lowp));
    // slots that took a new start in the last sweep have a dense x (the gather skips them)
    if (otf) RC(sweep_u_dense(h, engine, r, &cur->n_new, &cur->n_new, r, false, h->new_slot));
    if (pl.union_in) RC(sweep_u_union(h, S, cur, r));
    CK(timed(h, SPCA_K_U_SPARSE, 1, [&] {
      if (h->sparse)
        return launch_spmv_support(sp_cols(h), n, h->sup_idx, h->sup_val, p, S, r, h->U, h->ldU, &cur->use_gather,
                                   st);
      if (pl.lowp && f8_sweeps(h))
        return launch_gemm1_sparse_f8(h->AT8, h->ldAT8, h->at8_inv, n, h->sup_idx, h->sup_val, p, S, r, h->U, h->ldU,
                                      &cur->use_gather, st);
      if (pl.lowp)
        return launch_gemm1_sparse_lowp(h->ATpl, h->ldAT, h->at_inv, n, h->sup_idx, h->sup_val, p, S, r, h->U, h->ldU,
                                        &cur->use_gather, st);
      return launch_gemm1_sparse(h->AT32, h->ldAT, n, h->sup_idx, h->sup_val, p, S, r, h->U, h->ldU,
                                 &cur->use_gather, st);
    }));
    // deflated sparse A: u -= W (Z^T x)
    RC(sweep_lowrank_u(h, r, &cur->active, h->act));
    // y-step, v = A^T y
    RC(sweep_y_v(h, engine, form, r, S, &cur->active, r, pl.lowp));
    CK(cudaMemsetAsync(nxt, 0, sizeof(Ctrl), st));
    XstepArgs xk = xa;
    xk.sparse_cap = pl.sparse_cap;
    CK(timed(h, SPCA_K_XSTEP, 3, [&] {   // candidate filter and operator, full x-step
      return launch_xstep(xk, h->V, h->ldX, r, h->X, h->ldX, S, h->sup_idx, h->sup_val, nxt, h->xs, st);
    }));
    if (otf) {
      // stopped slots: archive their start, give them the next starts (Section 4.3)
      CK(timed(h, SPCA_K_INIT, 3, [&] {
        cudaError_t e = launch_otf_retire(r, l, S, h->slot_start, h->next_start, h->arc, h->retire_slot,
                                          h->retire_start, h->new_slot, nxt, h->X, h->ldX, p, st);
        if (e != cudaSuccess) return e;
        return launch_start_init(x0src, ld0, P.seed, r, p, h->X, h->ldX, S, gamma0, h->new_slot, h->slot_start,
                                 &nxt->n_new, st);
      }));
    }
    CK(timed(h, SPCA_K_XSTEP, 1, [&] {   // the active list of the next sweep
      return launch_active_list(h->status, h->nnz, r, h->act, h->rank, nxt, st);
    }));
    if (pl.union_out) {
      CK(timed(h, SPCA_K_U_SPARSE, 2, [&] {
        return launch_union(h->sup_idx, p, S, r, p, h->mark, h->colpos, h->collist, h->kcap, nxt, st);
      }));
    }
    return SPCA_OK;
  };
  // captured segments live in the handle and are reused by later solves with the same
  // parameters (every argument their kernels were captured with is in the key)
  std::vector<SegGraph> &graphs = h->graphs;
  if (h->graph_gen != h->ws_gen || h->graph_prof != h->prof_mask) {
    release_graphs(h);
    h->graph_gen = h->ws_gen;
    h->graph_prof = h->prof_mask;
  }
  if (graphs.size() > 64) release_graphs(h);
  auto bits = [](double d) {
    int64_t b;
    memcpy(&b, &d, sizeof b);
    return b;
  };
  const std::vector<int> solve_key = {form, engine, r, l, (int)(x0src != nullptr), max_iter, C, L, F0, (int)target,
                                      h->defl_k,
                                      (int)(bits(P.s) & 0xffffffff), (int)(bits(P.s) >> 32),
                                      (int)(bits(P.gamma) & 0xffffffff), (int)(bits(P.gamma) >> 32),
                                      (int)(bits(P.tol) & 0xffffffff), (int)(bits(P.tol) >> 32),
                                      // on-the-fly replacement reads x0 and the seed in the sweeps
                                      (int)(otf ? (reinterpret_cast<uintptr_t>(x0src) & 0xffffffffu) : 0),
                                      (int)(otf ? (reinterpret_cast<uintptr_t>(x0src) >> 32) : 0),
                                      (int)(otf ? (P.seed & 0xffffffffu) : 0), (int)(otf ? (P.seed >> 32) : 0)};
  std::vector<SweepPlan> plans;
  std::vector<int> key;
  int rc = SPCA_OK;
  // every start runs at most max_iter sweeps and every sweep advances at least one start, so l
  // starts end within l * max_iter sweeps (the loop stops as soon as no slot is active)
  const int max_total = otf ? (int)std::min<int64_t>((int64_t)l * max_iter, INT32_MAX / 2) : max_iter;
  // a small dense matrix on the CUDA-core engine: every sweep of every start in one launch, since
  // the chain of launches of a sweep, not its work, would set the time (AUTO only: an explicit
  // engine keeps the per-sweep kernels)
  const bool small = P.engine == SPCA_ENGINE_AUTO && engine == SPCA_ENGINE_SIMT && !h->sparse && !otf && L == 0 &&
                     h->defl_k == 0 && h->A32 && small_sweeps_fit(h->n, h->p, r);
  if (small) {
    CK(timed(h, SPCA_K_XSTEP, 1, [&] {
      return launch_small_sweeps(xa, h->A32, h->ldA, n, p, h->X, h->ldX, h->U, h->Y, h->ldU, h->V, S, h->sup_idx,
                                 h->sup_val, r, max_iter, st);
    }));
    if (P.timeout_us > 0 && std::chrono::duration_cast<std::chrono::microseconds>(
                                std::chrono::steady_clock::now() - t_start).count() > P.timeout_us) {
      CK(cudaStreamSynchronize(st));
      if (std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t_start).count() >
          P.timeout_us)
        return fail(h, SPCA_E_TIMEOUT, "the solve ran past timeout_us%s");
    }
  }
  for (int k0 = 1; k0 <= max_total && rc == SPCA_OK && !small;) {
    const int k1 = std::min(max_total, (k0 + check_every - 1) / check_every * check_every);
    plans.clear();
    key = solve_key;
    key.insert(key.end(), {k0 & 1, k1 - k0});
    for (int k = k0; k <= k1; ++k) {
      SweepPlan pl{};
      pl.k = k;
      // sweeps F0 + 1 .. F0 + L read the low-precision copy of A (the leading FP16 plane or E4M3)
      pl.lowp = k > F0 && k <= F0 + L;
      pl.dense_in = dense_queued;
      pl.union_in = union_built;
      dense_queued = max_nnz > sparse_cap / 2;
      pl.sparse_cap = dense_queued ? sparse_cap : p;   // p: the gather for every support
      const bool next_lowp = k + 1 > F0 && k + 1 <= F0 + L;
      union_built = engine == SPCA_ENGINE_TC && !otf && !all_lowp && !next_lowp && sum_nnz <= (int64_t)kUnionTry * h->kcap &&
                    h->n * sum_nnz >= kUnionMinReads;
      pl.union_out = union_built;
      plans.push_back(pl);
      key.insert(key.end(), {pl.lowp, pl.dense_in, pl.union_in, pl.union_out, pl.sparse_cap});
    }
    SegGraph *g = nullptr;
    for (SegGraph &c : graphs)
      if (c.key == key) g = &c;
    if (!g) {
      // capture this plan's kernels (relaxed mode: the launchers may set function attributes)
      graphs.emplace_back();
      g = &graphs.back();
      g->key = key;
      h->capturing = true;
      std::fill(std::begin(h->cap_counts), std::end(h->cap_counts), 0);
      h->cap_timings.clear();
      cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
      if (ce == cudaSuccess) {
        for (const SweepPlan &pl : plans)
          if ((rc = enqueue(pl)) != SPCA_OK) break;
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(st, &graph);
        if (ce == cudaSuccess) ce = ee;
        if (ce == cudaSuccess && rc == SPCA_OK) ce = cudaGraphInstantiate(&g->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
      }
      h->capturing = false;
      std::copy(std::begin(h->cap_counts), std::end(h->cap_counts), std::begin(g->counts));
      g->timings.swap(h->cap_timings);
      if (rc == SPCA_OK && ce != cudaSuccess) rc = fail(h, SPCA_E_CUDA, "CUDA error: %s", cudaGetErrorString(ce));
      if (rc != SPCA_OK) break;
    }
    if (cudaGraphLaunch(g->exec, st) != cudaSuccess) {
      rc = fail(h, SPCA_E_CUDA, "CUDA error: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    for (int q = 0; q < SPCA_K_COUNT; ++q) h->launches[q] += g->counts[q];
    Ctrl *last = h->ctrl + (k1 & 1);
    if (cudaMemcpyAsync(h->h_ctrl, last, sizeof(Ctrl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = fail(h, SPCA_E_CUDA, "CUDA error: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    for (auto &t : g->timings) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, std::get<1>(t), std::get<2>(t));
      h->ms[std::get<0>(t)] += ms;
    }
    if (h->h_ctrl->active == 0) break;
    if (P.timeout_us > 0 &&
        std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t_start).count() >
            P.timeout_us) {
      rc = fail(h, SPCA_E_TIMEOUT, "the solve ran past timeout_us%s");
      break;
    }
    nhost = h->h_ctrl->active;   // counts only fall: any earlier value stays an upper bound
    sum_nnz = h->h_ctrl->sum_nnz;
    max_nnz = h->h_ctrl->max_nnz;
    k0 = k1 + 1;
  }
  RC(rc);
  RC(read_dev_err(h));

  // ---- a7: FP64-class objective, best start, y(x) and support of the best x
  if (h->sparse) {
    // u = A x by rows in compensated FP32 pairs, then f, the best start and its outputs
    OtfArchive view = h->arc;
    if (!otf) {
      view.x = h->X;
      view.U = h->U;
      view.gamma = S.gamma;
      view.f = S.f;
      view.ev = S.ev;
    }
    const int cnt = otf ? l : r;
    double *part = otf ? h->otf_partials : h->partials;
    CK(timed(h, SPCA_K_FINALISE, 4, [&] {
      // the support lists are kept for a plain solve's starts (on-the-fly replacement archives x only);
      // after deflation u is A_k x = A x - W (Z^T x)
      const LowRank L = low_rank(h);
      cudaError_t e = launch_lowrank_coef(view.x, h->ldX, p, nullptr, nullptr, cnt, L.Z, L.ldz, L.k, L.coef, st);
      if (e == cudaSuccess)
        e = launch_fin_csr(sp_rows(h), sp_cols(h), view.x, h->ldX, cnt, otf ? nullptr : S.nnz,
                           otf ? nullptr : h->sup_idx, otf ? nullptr : h->sup_val, p, h->Bt, h->ldb, view.U, h->ldU,
                           part, L, st);
      if (e == cudaSuccess) e = launch_objective_reduce(form, part, (n + 255) / 256, p, view, cnt, h->ldX, st);
      StartState Sa{};
      Sa.f = view.f;
      Sa.ev = view.ev;
      if (e == cudaSuccess) e = launch_best(form, target ? 1 : 0, Sa, cnt, h->best, st);
      if (e == cudaSuccess)
        e = launch_best_outputs(form, h->best, view.U, h->ldU, n, view.x, h->ldX, p, h->y_out, h->x_out,
                                h->support_out, h->nnz_out, st);
      return e;
    }));
  } else if (otf) {
    CK(timed(h, SPCA_K_FINALISE, 4, [&] {
      cudaError_t e = launch_otf_objectives(form, h->AT32, h->ldAT, n, p, h->arc, l, h->ldX, h->ldU,
                                            h->otf_partials, st);
      StartState Sa{};
      Sa.f = h->arc.f;
      Sa.ev = h->arc.ev;
      if (e == cudaSuccess) e = launch_best(form, target ? 1 : 0, Sa, l, h->best, st);
      if (e == cudaSuccess)
        e = launch_best_outputs(form, h->best, h->arc.U, h->ldU, n, h->arc.x, h->ldX, p, h->y_out, h->x_out,
                                h->support_out, h->nnz_out, st);
      return e;
    }));
  } else {
    CK(timed(h, SPCA_K_FINALISE, 4, [&] {
      cudaError_t e =
          h->resident16
              ? launch_finalise_h(form, static_cast<const __half *>(h->ATpl), h->at_inv, h->ldAT, n, S, r, h->U,
                                  h->ldU, h->sup_idx, h->sup_val, p, h->partials, st)
              : launch_finalise(form, h->AT32, h->ldAT, n, p, h->X, h->ldX, S, r, h->U, h->ldU, h->sup_idx,
                                h->sup_val, p, h->partials, st);
      if (e == cudaSuccess) e = launch_best(form, target ? 1 : 0, S, r, h->best, st);
      if (e == cudaSuccess)
        e = launch_best_outputs(form, h->best, h->U, h->ldU, n, h->X, h->ldX, p, h->y_out, h->x_out,
                                h->support_out, h->nnz_out, st);
      return e;
    }));
  }

  // ---- results to the host (the archive of all l starts with on-the-fly replacement)
  const int nres = l;
  const int *d_status = otf ? h->arc.status : h->status, *d_iters = otf ? h->arc.iters : h->iters;
  const double *d_f = otf ? h->arc.f : h->f, *d_ev = otf ? h->arc.ev : h->ev;
  const double *d_gam = otf ? h->arc.gamma : h->gamma, *d_F = otf ? h->arc.F : h->F;
  const float *d_x = otf ? h->arc.x : h->X;
  std::vector<int> status(nres), iters(nres);
  std::vector<double> f(nres), ev(nres), gam(nres), F(nres);
  int best = 0;
  int64_t nnz = 0;
  CK(cudaMemcpyAsync(status.data(), d_status, nres * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(iters.data(), d_iters, nres * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(f.data(), d_f, nres * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ev.data(), d_ev, nres * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(gam.data(), d_gam, nres * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(F.data(), d_F, nres * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&best, h->best, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&nnz, h->nnz_out, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (res->x) CK(cudaMemcpyAsync(res->x, h->x_out, (size_t)p * sizeof(float), cudaMemcpyDeviceToHost, st));
  if (res->y) CK(cudaMemcpyAsync(res->y, h->y_out, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, st));
  if (res->support && nnz > 0)
    CK(cudaMemcpyAsync(res->support, h->support_out, (size_t)nnz * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  if (res->start_x)
    CK(cudaMemcpy2DAsync(res->start_x, (size_t)p * sizeof(float), d_x, h->ldX * sizeof(float),
                         (size_t)p * sizeof(float), nres, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));

  int64_t sweeps = 0;
  int nconv = 0, ndeg = 0;
  for (int c = 0; c < nres; ++c) {
    sweeps += iters[c];
    nconv += status[c] == SPCA_ST_CONVERGED;
    ndeg += status[c] == SPCA_ST_DEGENERATE;
  }
  res->objective = f[best];
  res->explained_variance = ev[best];
  res->gamma = is_pen(form) ? gam[best] : 0.0;
  res->best_start = best;
  res->best_iters = iters[best];
  res->best_status = status[best];
  res->converged = nconv;
  res->degenerate = ndeg;
  res->sweeps_total = sweeps;
  res->nnz = nnz;
  if (res->start_objective) memcpy(res->start_objective, f.data(), nres * sizeof(double));
  if (res->start_explained) memcpy(res->start_explained, ev.data(), nres * sizeof(double));
  if (res->start_F) memcpy(res->start_F, F.data(), nres * sizeof(double));
  if (res->start_iters) memcpy(res->start_iters, iters.data(), nres * sizeof(int));
  if (res->start_status) memcpy(res->start_status, status.data(), nres * sizeof(int));
  if (res->start_gamma) {
    for (int c = 0; c < nres; ++c) res->start_gamma[c] = is_pen(form) ? gam[c] : 0.0;
  }
  return SPCA_OK;
}

}  // extern "C"
