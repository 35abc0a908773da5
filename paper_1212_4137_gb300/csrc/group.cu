// group.cu -- spca_solve_group: Algorithm 2 for many independent problems at once (each with its own
// matrix, formulation, s or gamma and starts), every phase of a sweep one launch over all of them:
// the dense u = A x of the first sweep and v = A^T y of every sweep as one persistent tensor-core
// launch over the tiles of all problems (k_gemm_grouped), the support gather, y-step, x-step and
// active lists as one launch each over all starts or problems.  The sweeps between two read-backs
// of the problems' control words are captured into a CUDA graph and replayed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "spca_handle.cuh"

using namespace spca;

namespace {

struct GroupGraph {
  uint64_t key = 0;
  cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct spca_group {
  cudaStream_t stream = nullptr;   // the group's own non-blocking stream (captured into graphs)
  cudaStream_t user = nullptr;     // the caller's stream: each solve starts after its prior work
  cudaEvent_t order_ev = nullptr;
  int sms = 1;
  char *ws = nullptr;              // device workspace, grown on demand
  size_t ws_bytes = 0;
  Ctrl *h_ctrl = nullptr;          // pinned mirror of one parity's control words
  int h_ctrl_cap = 0;
  int *h_err = nullptr;            // pinned mirror of the device error word
  std::vector<GroupGraph> graphs;  // captured sweep segments and finalisations
  char last_error[256] = {0};
};

namespace {

int gfail(spca_group *g, int code, const char *msg) {
  if (g) snprintf(g->last_error, sizeof(g->last_error), "%s", msg);
  return code;
}

#define GCK(expr)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      if (g) snprintf(g->last_error, sizeof(g->last_error), "CUDA error: %s", cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? SPCA_E_NOMEM : SPCA_E_CUDA;                 \
    }                                                                                      \
  } while (0)

// FNV-1a over bytes (keys of the captured graphs)
uint64_t fnv(uint64_t h, const void *p, size_t n) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

// bump allocator over the workspace: 256-byte aligned blocks
struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  }
};

// per-problem host bookkeeping
struct HostProb {
  spca_handle *h;
  spca_params P;
  const float *x0;
  spca_result *res;
  int r, n, p, start0, target, calib;
  int64_t ldX, ldU;
  size_t oX, oV, oU, oXpl, oYpl, oxs, oxi, osi, osv, opart, oyout, oxout, osup;
};

// the problem's parameters against Algorithm 2's requirements (as spca_solve checks them)
const char *check_problem(const spca_problem &q) {
  const spca_params &P = q.prm;
  const spca_handle *h = q.h;
  if (!h || !q.res) return "NULL handle or result";
  if (h->sparse) return "a grouped solve takes dense matrices";
  if (!h->tc_ok) return "a grouped solve needs tensor cores (sm_100+)";
  const int form = P.form;
  if (form < 1 || form > 8) return "form must be 1..8";
  if (!std::isfinite(P.s) || !std::isfinite(P.gamma) || !std::isfinite(P.tol)) return "s, gamma and tol must be finite";
  if (uses_T(form) && (P.s < 1.0 || P.s > (double)h->p || P.s != std::floor(P.s)))
    return "L0 constraint: s must be an integer in [1, p]";
  if (uses_lam(form) && P.s < 1.0) return "L1 constraint: s must be >= 1";
  if (is_pen(form)) {
    if (P.gamma_mode != SPCA_GAMMA_FIXED && P.gamma_mode != SPCA_GAMMA_TARGET_NNZ) return "unknown gamma_mode";
    if (P.gamma_mode == SPCA_GAMMA_FIXED && P.gamma < 0.0) return "gamma must be >= 0";
    if (P.gamma_mode == SPCA_GAMMA_TARGET_NNZ &&
        (P.s < 1.0 || P.s > (double)h->p || P.s != std::floor(P.s) || P.gamma_calib_sweeps < 1))
      return "target mode: s must be an integer in [1, p] and gamma_calib_sweeps >= 1";
  }
  if (P.r < 1 || P.r > kMaxStarts || P.max_iter < 1) return "r must be in 1..65535 and max_iter >= 1";
  if (P.lowp_sweeps != 0 || P.total_starts > P.r || P.timeout_us < 0)
    return "a grouped solve runs FP32 sweeps from r starts (no lowp_sweeps, no total_starts)";
  if (P.engine != SPCA_ENGINE_AUTO && P.engine != SPCA_ENGINE_TC) return "a grouped solve runs on the tensor cores";
  return nullptr;
}

}  // namespace

extern "C" {

int spca_group_create(spca_group **out, void *cuda_stream) {
  if (!out) return SPCA_E_INVALID;
  int ndev = 0, dev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1 || cudaGetDevice(&dev) != cudaSuccess) return SPCA_E_CUDA;
  spca_group *g = new (std::nothrow) spca_group();
  if (!g) return SPCA_E_NOMEM;
  g->user = static_cast<cudaStream_t>(cuda_stream);
  if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->order_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaMallocHost((void **)&g->h_err, sizeof(int)) != cudaSuccess) {
    spca_group_destroy(g);
    return SPCA_E_CUDA;
  }
  *out = g;
  return SPCA_OK;
}

void spca_group_destroy(spca_group *g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (GroupGraph &q : g->graphs)
    if (q.exec) cudaGraphExecDestroy(q.exec);
  if (g->ws) cudaFree(g->ws);
  if (g->h_ctrl) cudaFreeHost(g->h_ctrl);
  if (g->h_err) cudaFreeHost(g->h_err);
  if (g->order_ev) cudaEventDestroy(g->order_ev);
  if (g->stream) cudaStreamDestroy(g->stream);
  delete g;
}

const char *spca_group_last_error(const spca_group *g) { return g ? g->last_error : ""; }

int spca_solve_group(spca_group *g, spca_problem *probs, int count, const spca_group_tiles *tiles) {
  if (!g || !probs || count < 1) return gfail(g, SPCA_E_INVALID, "NULL group or problems, or count < 1");
  if (count > kGroupMaxTasks) return gfail(g, SPCA_E_UNSUPPORTED, "more than 1024 problems in one group");
  int bn = 64, stages = 4;
  if (tiles && (tiles->tile_n || tiles->stages)) {
    bn = tiles->tile_n;
    stages = tiles->stages;
    if (!grouped_config_ok(bn, stages)) return gfail(g, SPCA_E_INVALID, "unknown tile shape (tile_n, stages)");
  }
  for (int i = 0; i < count; ++i)
    if (const char *bad = check_problem(probs[i])) return gfail(g, SPCA_E_INVALID, bad);
  cudaStream_t st = g->stream;
  GCK(cudaEventRecord(g->order_ev, g->user));
  GCK(cudaStreamWaitEvent(st, g->order_ev, 0));

  // ---- layout of the workspace
  std::vector<HostProb> hp(count);
  Layout L;
  int64_t R = 0;
  int max_n = 1, max_p = 1, max_iter = 1;
  for (int i = 0; i < count; ++i) {
    HostProb &q = hp[i];
    q.h = probs[i].h;
    q.P = probs[i].prm;
    q.x0 = probs[i].x0;
    q.res = probs[i].res;
    q.r = q.P.r;
    q.n = (int)q.h->n;
    q.p = (int)q.h->p;
    q.start0 = (int)R;
    q.target = is_pen(q.P.form) && q.P.gamma_mode == SPCA_GAMMA_TARGET_NNZ;
    q.calib = q.target ? q.P.gamma_calib_sweeps : 0;
    q.ldX = pad_ld(q.p);
    q.ldU = pad_ld(q.n);
    R += q.r;
    max_n = std::max(max_n, q.n);
    max_p = std::max(max_p, q.p);
    max_iter = std::max(max_iter, q.P.max_iter);
  }
  if (R > INT32_MAX / 2) return gfail(g, SPCA_E_UNSUPPORTED, "too many starts in one group");
  const size_t o_prob = L.take(sizeof(GProb) * count);
  const size_t o_map = L.take(sizeof(CUtensorMap) * 4 * count);   // A planes, A^T planes, X planes, Y planes
  const size_t o_task = L.take(sizeof(GTask) * 3 * count);        // u (first sweep), v for each parity
  const size_t o_start_prob = L.take(sizeof(int) * R);
  const size_t o_ctrl = L.take(sizeof(Ctrl) * 2 * count);         // parity-major
  const size_t o_best = L.take(sizeof(int) * count);
  const size_t o_nnzout = L.take(sizeof(int64_t) * count);
  const size_t o_err = L.take(sizeof(int));
  const size_t o_status = L.take(sizeof(int) * R), o_iters = L.take(sizeof(int) * R), o_nnz = L.take(sizeof(int) * R);
  const size_t o_F = L.take(8 * R), o_Fp = L.take(8 * R), o_gam = L.take(8 * R), o_f = L.take(8 * R), o_ev = L.take(8 * R);
  const size_t o_thr = L.take(4 * R), o_tprev = L.take(4 * R), o_xfast = L.take(4 * R);
  const size_t o_act = L.take(sizeof(int) * R), o_rank = L.take(sizeof(int) * R);
  const size_t zero_from = L.off;   // the vector blocks below start zeroed (padded columns)
  for (HostProb &q : hp) {
    q.oX = L.take(4 * (size_t)q.r * q.ldX);
    q.oV = L.take(4 * (size_t)q.r * q.ldX);
    q.oU = L.take(4 * (size_t)q.r * q.ldU);
    q.oXpl = L.take(2 * 2 * (size_t)q.r * q.ldX);
    q.oYpl = L.take(2 * 2 * (size_t)q.r * q.ldU);
  }
  const size_t zero_to = L.off;
  for (HostProb &q : hp) {
    q.oxs = L.take(4 * (size_t)q.r);
    q.oxi = L.take(4 * (size_t)q.r);
    q.osi = L.take(4 * (size_t)q.r * q.p);
    q.osv = L.take(4 * (size_t)q.r * q.p);
    q.opart = L.take(16 * (size_t)q.r * ((q.n + 255) / 256));
    q.oyout = L.take(4 * (size_t)q.ldU);
    q.oxout = L.take(4 * (size_t)q.ldX);
    q.osup = L.take(8 * (size_t)q.p);
  }
  if (L.off > g->ws_bytes) {
    GCK(cudaStreamSynchronize(st));
    for (GroupGraph &q : g->graphs)
      if (q.exec) cudaGraphExecDestroy(q.exec);
    g->graphs.clear();
    if (g->ws) cudaFree(g->ws);
    g->ws = nullptr;
    g->ws_bytes = 0;
    GCK(cudaMalloc((void **)&g->ws, L.off));
    g->ws_bytes = L.off;
  }
  if (g->h_ctrl_cap < count) {
    if (g->h_ctrl) cudaFreeHost(g->h_ctrl);
    g->h_ctrl = nullptr;
    g->h_ctrl_cap = 0;
    GCK(cudaMallocHost((void **)&g->h_ctrl, sizeof(Ctrl) * count));
    g->h_ctrl_cap = count;
  }
  char *W = g->ws;
  auto at = [&](size_t o) { return W + o; };
  GProb *dP = reinterpret_cast<GProb *>(at(o_prob));
  CUtensorMap *dmaps = reinterpret_cast<CUtensorMap *>(at(o_map));
  GTask *dtasks = reinterpret_cast<GTask *>(at(o_task));
  int *d_start_prob = reinterpret_cast<int *>(at(o_start_prob));
  Ctrl *dctrl = reinterpret_cast<Ctrl *>(at(o_ctrl));
  int *dbest = reinterpret_cast<int *>(at(o_best));
  int64_t *dnnzout = reinterpret_cast<int64_t *>(at(o_nnzout));
  int *derr = reinterpret_cast<int *>(at(o_err));
  StartState all{};
  all.status = reinterpret_cast<int *>(at(o_status));
  all.iters = reinterpret_cast<int *>(at(o_iters));
  all.nnz = reinterpret_cast<int *>(at(o_nnz));
  all.F = reinterpret_cast<double *>(at(o_F));
  all.F_prev = reinterpret_cast<double *>(at(o_Fp));
  all.gamma = reinterpret_cast<double *>(at(o_gam));
  all.f = reinterpret_cast<double *>(at(o_f));
  all.ev = reinterpret_cast<double *>(at(o_ev));
  all.thr = reinterpret_cast<float *>(at(o_thr));
  all.tprev = reinterpret_cast<float *>(at(o_tprev));
  all.xfast = reinterpret_cast<int *>(at(o_xfast));
  int *dact = reinterpret_cast<int *>(at(o_act)), *drank = reinterpret_cast<int *>(at(o_rank));
  GCK(cudaMemsetAsync(at(zero_from), 0, zero_to - zero_from, st));
  GCK(cudaMemsetAsync(derr, 0, sizeof(int), st));
  GCK(cudaMemsetAsync(dctrl, 0, sizeof(Ctrl) * 2 * count, st));

  // ---- problem table, tensor maps, tile tasks
  std::vector<GProb> P(count);
  std::vector<CUtensorMap> maps(4 * count);
  std::vector<int> start_prob(R);
  for (int i = 0; i < count; ++i) {
    HostProb &q = hp[i];
    GProb &d = P[i];
    d.n = q.n;
    d.p = q.p;
    d.r = q.r;
    d.start0 = q.start0;
    d.form = q.P.form;
    d.ldX = q.ldX;
    d.ldU = q.ldU;
    d.ldAT = q.h->ldAT;
    d.AT32 = q.h->AT32;
    d.X = reinterpret_cast<float *>(at(q.oX));
    d.V = reinterpret_cast<float *>(at(q.oV));
    d.U = reinterpret_cast<float *>(at(q.oU));
    d.Xpl = reinterpret_cast<__half *>(at(q.oXpl));
    d.Ypl = reinterpret_cast<__half *>(at(q.oYpl));
    d.xps = (int64_t)q.r * q.ldX;
    d.yps = (int64_t)q.r * q.ldU;
    d.x_scale = reinterpret_cast<float *>(at(q.oxs));
    d.x_inv = reinterpret_cast<float *>(at(q.oxi));
    d.sup_idx = reinterpret_cast<int *>(at(q.osi));
    d.sup_val = reinterpret_cast<float *>(at(q.osv));
    d.act = dact + q.start0;
    d.rank = drank + q.start0;
    d.ctrl[0] = dctrl + i;
    d.ctrl[1] = dctrl + count + i;
    StartState s = all;
    s.status += q.start0; s.iters += q.start0; s.nnz += q.start0;
    s.F += q.start0; s.F_prev += q.start0; s.gamma += q.start0; s.f += q.start0; s.ev += q.start0;
    s.thr += q.start0; s.tprev += q.start0; s.xfast += q.start0;
    d.st = s;
    XstepArgs &a = d.xa;
    a = XstepArgs{};
    a.form = q.P.form;
    a.p = q.p;
    a.s = q.P.s;
    a.thr_fixed = uses_U(q.P.form) ? u_threshold(q.P.gamma) : (float)q.P.gamma;
    a.gamma_fixed = q.P.gamma;
    a.tol = q.P.tol;
    a.max_iter = q.P.max_iter;
    a.cap = q.p;
    a.sparse_cap = q.p;   // the support gather serves every support after the first sweep
    a.schedule = 1;
    a.target = q.target;
    a.calib_sweeps = q.calib;
    a.lowp_sweeps = 0;
    a.stop_enabled = q.P.tol >= 0.0 ? 1 : 0;
    d.ld0 = q.ldX;
    d.x0 = nullptr;
    d.key = 0;
    if (q.x0) {
      // the given starts, copied into X and normalised there
      d.x0 = d.X;
      GCK(cudaMemcpy2DAsync(d.X, q.ldX * sizeof(float), q.x0, (size_t)q.p * sizeof(float), (size_t)q.p * sizeof(float),
                            q.r, q.P.x0_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else {
      auto mixh = [](uint64_t z) {
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
      };
      d.key = mixh(q.P.seed ^ mixh(5ull));   // the starts' stream of the single solve
    }
    d.gamma0 = is_pen(q.P.form) && !q.target ? q.P.gamma : 0.0;
    for (int c = 0; c < q.r; ++c) start_prob[q.start0 + c] = i;
    maps[4 * i + 0] = q.h->pmA.m[0];
    maps[4 * i + 1] = q.h->pmAT.m[0];
    GCK(make_plane_map(&maps[4 * i + 2], d.Xpl, q.r, q.ldX, 2, 64, 64));
    GCK(make_plane_map(&maps[4 * i + 3], d.Ypl, q.r, q.ldU, 2, 64, 64));
  }
  // x0 must be finite (as spca_solve checks)
  {
    int *flag = derr;   // borrowed before the sweeps; zeroed again below
    for (int i = 0; i < count; ++i)
      if (hp[i].x0) GCK(launch_check_finite(P[i].X, hp[i].r, hp[i].p, hp[i].ldX, flag, st));
    GCK(cudaMemcpyAsync(g->h_err, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    GCK(cudaStreamSynchronize(st));
    if (*g->h_err) return gfail(g, SPCA_E_INVALID, "x0 has a non-finite entry");
    GCK(cudaMemsetAsync(derr, 0, sizeof(int), st));
  }
  // tile tasks: u = A x (first sweep) and v = A^T y (per parity), each list ordered by falling K
  std::vector<GTask> tasks(3 * count);
  int total_u = 0, total_v = 0;
  auto build = [&](int which, int parity, int *total) {
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    auto kb = [&](int i) { return which == 0 ? (hp[i].p + 63) / 64 : (hp[i].n + 63) / 64; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return kb(a) > kb(b); });
    GTask *base = tasks.data() + (which == 0 ? 0 : (1 + parity) * count);
    int t0 = 0;
    for (int k = 0; k < count; ++k) {
      const int i = order[k];
      const HostProb &q = hp[i];
      GTask &T = base[k];
      T = GTask{};
      const bool u = which == 0;
      T.pmap = dmaps + 4 * i + (u ? 0 : 1);
      T.qmap = dmaps + 4 * i + (u ? 2 : 3);
      T.M = u ? q.n : q.p;
      T.kblocks = kb(i);
      T.nmax = q.r;
      T.nb = u || !is_l1_var(q.P.form) ? 2 : 1;
      T.n_dev = &P[i].ctrl[parity]->active;
      T.col_map = P[i].act;
      T.out = u ? P[i].U : P[i].V;
      T.ldo = u ? q.ldU : q.ldX;
      T.row_inv = u ? q.h->a_inv : q.h->at_inv;
      T.col_inv = u ? P[i].x_inv : nullptr;
      T.q_inv = u ? 1.0f : kQInv;
      T.pairs = u || !is_l1_var(q.P.form) ? pairs_general() : pairs_sign();
      T.mt = (T.M + TC_BM_ROWS - 1) / TC_BM_ROWS;
      T.nt = (q.r + bn - 1) / bn;
      T.tile0 = t0;
      t0 += T.mt * T.nt;
    }
    *total = t0;
  };
  build(0, 0, &total_u);   // the first sweep reads parity 0
  build(1, 0, &total_v);
  build(1, 1, &total_v);
  GCK(cudaMemcpyAsync(dP, P.data(), sizeof(GProb) * count, cudaMemcpyHostToDevice, st));
  GCK(cudaMemcpyAsync(dmaps, maps.data(), sizeof(CUtensorMap) * 4 * count, cudaMemcpyHostToDevice, st));
  GCK(cudaMemcpyAsync(dtasks, tasks.data(), sizeof(GTask) * 3 * count, cudaMemcpyHostToDevice, st));
  GCK(cudaMemcpyAsync(d_start_prob, start_prob.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
  const uint64_t wait_ns = 2000000000ull;

  // ---- starts, active lists of the first sweep
  GCK(launch_g_start_init(dP, d_start_prob, (int)R, st));
  GCK(launch_g_active(dP, count, 0, st));

  // ---- the sweeps, in captured segments of up to 4 between read-backs
  uint64_t skey = 1469598103934665603ull;
  skey = fnv(skey, P.data(), sizeof(GProb) * count);
  skey = fnv(skey, tasks.data(), sizeof(GTask) * 3 * count);
  skey = fnv(skey, &bn, sizeof bn);
  skey = fnv(skey, &stages, sizeof stages);
  if (g->graphs.size() > 32) {
    GCK(cudaStreamSynchronize(st));
    for (GroupGraph &q : g->graphs)
      if (q.exec) cudaGraphExecDestroy(q.exec);
    g->graphs.clear();
  }
  auto enqueue_sweep = [&](int k) -> cudaError_t {
    const int cur = (k - 1) & 1, nxt = k & 1;
    cudaError_t e;
    if (k == 1) {
      e = launch_g_xplanes(dP, d_start_prob, (int)R, st);
      if (e == cudaSuccess) e = launch_gemm_grouped(dtasks, count, total_u, bn, stages, g->sms, derr, wait_ns, st);
    } else {
      e = launch_g_gather(dP, d_start_prob, (int)R, max_n, st);
    }
    if (e == cudaSuccess) e = launch_g_ystep(dP, d_start_prob, (int)R, st);
    if (e == cudaSuccess)
      e = launch_gemm_grouped(dtasks + (1 + cur) * count, count, total_v, bn, stages, g->sms, derr, wait_ns, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dctrl + nxt * count, 0, sizeof(Ctrl) * count, st);
    if (e == cudaSuccess) e = launch_g_xstep(dP, d_start_prob, (int)R, max_p, nxt, g->sms, st);
    if (e == cudaSuccess) e = launch_g_active(dP, count, nxt, st);
    return e;
  };
  auto run_captured = [&](uint64_t key, auto &&body) -> int {
    GroupGraph *gg = nullptr;
    for (GroupGraph &q : g->graphs)
      if (q.key == key) gg = &q;
    if (!gg) {
      g->graphs.emplace_back();
      gg = &g->graphs.back();
      gg->key = key;
      cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
      cudaError_t be = cudaSuccess;
      if (ce == cudaSuccess) {
        be = body();
        cudaGraph_t graph = nullptr;
        ce = cudaStreamEndCapture(st, &graph);
        if (ce == cudaSuccess && be == cudaSuccess) ce = cudaGraphInstantiate(&gg->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
      }
      if (be != cudaSuccess) ce = be;
      if (ce != cudaSuccess) {
        g->graphs.pop_back();
        GCK(ce);
      }
    }
    GCK(cudaGraphLaunch(gg->exec, st));
    return SPCA_OK;
  };
  const int check_every = 4;
  for (int k0 = 1; k0 <= max_iter;) {
    const int k1 = std::min(max_iter, k0 + check_every - 1);
    uint64_t key = fnv(skey, &k0, sizeof k0);
    key = fnv(key, &k1, sizeof k1);
    const int rc = run_captured(key, [&]() -> cudaError_t {
      for (int k = k0; k <= k1; ++k) {
        cudaError_t e = enqueue_sweep(k);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    });
    if (rc != SPCA_OK) return rc;
    GCK(cudaMemcpyAsync(g->h_ctrl, dctrl + (k1 & 1) * count, sizeof(Ctrl) * count, cudaMemcpyDeviceToHost, st));
    GCK(cudaStreamSynchronize(st));
    int64_t active = 0;
    for (int i = 0; i < count; ++i) active += g->h_ctrl[i].active;
    if (active == 0) break;
    k0 = k1 + 1;
  }
  GCK(cudaMemcpyAsync(g->h_err, derr, sizeof(int), cudaMemcpyDeviceToHost, st));
  GCK(cudaStreamSynchronize(st));
  if (*g->h_err) return gfail(g, *g->h_err, "a device-side wait timed out");

  // ---- the Table 1 objective of every start, the best start of each problem and its outputs
  const int rc = run_captured(fnv(skey, "fin", 3), [&]() -> cudaError_t {
    for (int i = 0; i < count; ++i) {
      const HostProb &q = hp[i];
      const GProb &d = P[i];
      cudaError_t e = launch_finalise(q.P.form, q.h->AT32, q.h->ldAT, q.n, q.p, d.X, q.ldX, d.st, q.r, d.U, q.ldU,
                                      d.sup_idx, d.sup_val, q.p, reinterpret_cast<double *>(at(q.opart)), st);
      if (e == cudaSuccess) e = launch_best(q.P.form, q.target, d.st, q.r, dbest + i, st);
      if (e == cudaSuccess)
        e = launch_best_outputs(q.P.form, dbest + i, d.U, q.ldU, q.n, d.X, q.ldX, q.p,
                                reinterpret_cast<float *>(at(q.oyout)), reinterpret_cast<float *>(at(q.oxout)),
                                reinterpret_cast<int64_t *>(at(q.osup)), dnnzout + i, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  });
  if (rc != SPCA_OK) return rc;

  // ---- results to the host
  std::vector<int> status(R), iters(R), best(count);
  std::vector<double> f(R), ev(R), gam(R), F(R);
  std::vector<int64_t> nnz(count);
  GCK(cudaMemcpyAsync(status.data(), all.status, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
  GCK(cudaMemcpyAsync(iters.data(), all.iters, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
  GCK(cudaMemcpyAsync(f.data(), all.f, 8 * R, cudaMemcpyDeviceToHost, st));
  GCK(cudaMemcpyAsync(ev.data(), all.ev, 8 * R, cudaMemcpyDeviceToHost, st));
  GCK(cudaMemcpyAsync(gam.data(), all.gamma, 8 * R, cudaMemcpyDeviceToHost, st));
  GCK(cudaMemcpyAsync(F.data(), all.F, 8 * R, cudaMemcpyDeviceToHost, st));
  GCK(cudaMemcpyAsync(best.data(), dbest, sizeof(int) * count, cudaMemcpyDeviceToHost, st));
  GCK(cudaMemcpyAsync(nnz.data(), dnnzout, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, st));
  GCK(cudaStreamSynchronize(st));
  for (int i = 0; i < count; ++i) {
    const HostProb &q = hp[i];
    spca_result *res = q.res;
    if (res->x) GCK(cudaMemcpyAsync(res->x, at(q.oxout), (size_t)q.p * 4, cudaMemcpyDeviceToHost, st));
    if (res->y) GCK(cudaMemcpyAsync(res->y, at(q.oyout), (size_t)q.n * 4, cudaMemcpyDeviceToHost, st));
    if (res->support && nnz[i] > 0)
      GCK(cudaMemcpyAsync(res->support, at(q.osup), (size_t)nnz[i] * 8, cudaMemcpyDeviceToHost, st));
    if (res->start_x)
      GCK(cudaMemcpy2DAsync(res->start_x, (size_t)q.p * 4, at(q.oX), q.ldX * 4, (size_t)q.p * 4, q.r,
                            cudaMemcpyDeviceToHost, st));
  }
  GCK(cudaStreamSynchronize(st));
  for (int i = 0; i < count; ++i) {
    const HostProb &q = hp[i];
    spca_result *res = q.res;
    const int b = best[i], o = q.start0;
    int64_t sweeps = 0;
    int nconv = 0, ndeg = 0;
    for (int c = 0; c < q.r; ++c) {
      sweeps += iters[o + c];
      nconv += status[o + c] == SPCA_ST_CONVERGED;
      ndeg += status[o + c] == SPCA_ST_DEGENERATE;
    }
    res->objective = f[o + b];
    res->explained_variance = ev[o + b];
    res->gamma = is_pen(q.P.form) ? gam[o + b] : 0.0;
    res->best_start = b;
    res->best_iters = iters[o + b];
    res->best_status = status[o + b];
    res->converged = nconv;
    res->degenerate = ndeg;
    res->sweeps_total = sweeps;
    res->nnz = nnz[i];
    for (int c = 0; c < q.r; ++c) {
      if (res->start_objective) res->start_objective[c] = f[o + c];
      if (res->start_explained) res->start_explained[c] = ev[o + c];
      if (res->start_F) res->start_F[c] = F[o + c];
      if (res->start_iters) res->start_iters[c] = iters[o + c];
      if (res->start_status) res->start_status[c] = status[o + c];
      if (res->start_gamma) res->start_gamma[c] = is_pen(q.P.form) ? gam[o + c] : 0.0;
    }
  }
  return SPCA_OK;
}

}  // extern "C"
