// group.cu -- groups of problems: Algorithm 2 for many independent problems at once (each with its
// own matrix, formulation, s or gamma and starts), every phase of a sweep one launch over all of
// them: the dense u = A x of a problem's first sweep and v = A^T y of every sweep as one persistent
// tensor-core launch over the tiles of all problems (k_gemm_grouped), the support gather, y-step,
// x-step and active lists as one launch each over all starts or problems.
//
// A group is a session: problems are admitted between segments of sweeps (each into a block of
// device memory of its own), every member sweeps in the same launches (a new member's first sweep,
// with its dense u = A x, beside the others' later ones), and a member whose starts have all
// stopped is finalised (Table 1 objective, best start, its outputs) and retired at the end of the
// segment.  spca_solve_group admits a whole set and steps it to the end with every segment
// captured into a CUDA graph; spca_group_admit / spca_group_step serve requests that arrive while
// others run (continuous batching at sweep boundaries).
#include <algorithm>
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

// bump allocator over a block: 256-byte aligned pieces
struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  }
};

// one admitted problem: its request, its block of device memory and its table entry
struct Member {
  spca_handle *h = nullptr;
  spca_params P{};
  spca_result *res = nullptr;
  int tag = 0;
  int r = 0, n = 0, p = 0, target = 0;
  int64_t ldX = 0, ldU = 0;
  char *mem = nullptr;            // the member's device block
  GProb d{};                      // its table entry (start0 set when the table is built)
  CUtensorMap *maps = nullptr;    // device: A planes, A^T planes, X planes
  double *partials = nullptr;
  float *y_out = nullptr, *x_out = nullptr;
  int64_t *support_out = nullptr, *nnz_out = nullptr;
  int *best = nullptr;
  bool first_pending = true;      // its first sweep (the dense u = A x) is still to run
};

uint64_t fnv(uint64_t h, const void *p, size_t n) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

}  // namespace

struct spca_group {
  cudaStream_t stream = nullptr;   // the group's own non-blocking stream
  // the group's own stream-ordered memory pool (member blocks, pool buffers): it keeps what is
  // freed for the next admissions instead of returning it to the device at every synchronisation
  cudaMemPool_t mempool = nullptr;
  cudaStream_t user = nullptr;     // the caller's stream: each call starts after its prior work
  cudaEvent_t order_ev = nullptr;
  int sms = 1;
  std::vector<Member> members;     // admitted, unfinished problems
  int64_t k = 0;                   // sweeps run so far (the parity of the control words)
  // the tables of the current members (device), grown on demand
  char *tab = nullptr;
  size_t tab_bytes = 0;
  GProb *dP = nullptr;
  int *d_start_prob = nullptr, *d_active = nullptr;
  GTask *d_tasks = nullptr;
  int2 *d_tiles[3] = {nullptr, nullptr, nullptr};   // tile lists: u, v of parity 0, v of parity 1
  int R = 0, total_u = 0, total_v = 0, n_u = 0, max_n = 1, max_p = 1, max_p_small = 0;
  bool any_large_p = false;
  bool tables_ok = false;
  // pools (members on one matrix that share v = A^T y): the table, its member list, and one
  // device block with each pool's V rows and Y planes (scratch of a sweep, rebuilt with the
  // tables; kept when the pools' shapes are unchanged)
  GPool *d_pools = nullptr;
  int *d_pool_members = nullptr;
  int npool = 0;
  char *pool_mem = nullptr;
  std::vector<int64_t> pool_sig;
  // the candidate x-step's scratch (per start: kXstepCand values and indices, one int4), grown
  // with the number of starts; used when some member's v is long enough (kCandMinP)
  char *cand_mem = nullptr;
  int cand_cap = 0;
  bool use_cand = false;
  int *h_active = nullptr;         // pinned: active counts at a segment's end
  int h_active_cap = 0;
  int *h_err = nullptr;            // pinned: the device error word
  int *d_err = nullptr;
  int bn = 64, stages = 4;
  bool tiles_auto = true;          // the shape follows the widest pool (spca_group_set_tiles)
  bool lowp_all = false;           // every member is a resident 16-bit matrix's (leading planes only)
  std::vector<GroupGraph> graphs;
  // staging of finished members' results: device buffer, pinned host mirror, copy descriptors
  char *stage_d = nullptr, *stage_h = nullptr;
  size_t stage_bytes = 0;
  CopyDesc *desc_d = nullptr;
  size_t desc_bytes = 0;
  char last_error[256] = {0};
};

namespace {

int gfail(spca_group *g, int code, const char *msg) {
  if (g) snprintf(g->last_error, sizeof(g->last_error), "%s", msg);
  return code;
}

#define GCK(expr)                                                                                     \
  do {                                                                                                \
    cudaError_t e_ = (expr);                                                                          \
    if (e_ != cudaSuccess) {                                                                          \
      if (g) snprintf(g->last_error, sizeof(g->last_error), "CUDA error: %s", cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? SPCA_E_NOMEM : SPCA_E_CUDA;                            \
    }                                                                                                 \
  } while (0)

#define GRC(expr)                   \
  do {                              \
    int rc_ = (expr);               \
    if (rc_ != SPCA_OK) return rc_; \
  } while (0)

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
  if (h->resident16 && (P.lowp_first != 0 || P.refine_sweeps != 0))
    return "every sweep of a resident 16-bit handle is a low-precision sweep: lowp_first and refine_sweeps must be 0";
  if (P.engine != SPCA_ENGINE_AUTO && P.engine != SPCA_ENGINE_TC) return "a grouped solve runs on the tensor cores";
  return nullptr;
}

uint64_t seed_key(uint64_t seed) {
  auto mixh = [](uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  return mixh(seed ^ mixh(5ull));   // the starts' stream of the single solve
}

// device bytes of a member's block for r starts on an n x p matrix
size_t member_layout(Member &m, size_t *o) {
  Layout L;
  const size_t r = (size_t)m.r;
  o[0] = L.take(4 * r * m.ldX);              // X
  o[1] = L.take(0);                          // (V: the pool's rows)
  o[2] = L.take(4 * r * m.ldU);              // U
  o[3] = L.take(2 * 2 * r * m.ldX);          // X planes
  o[4] = L.take(0);                          // (Y planes: the pool's rows)
  o[5] = L.off;                              // (end of the zeroed part: padded columns)
  o[6] = L.take(4 * r);                      // x_scale
  o[7] = L.take(4 * r);                      // x_inv
  o[8] = L.take(4 * r * m.p);                // sup_idx
  o[9] = L.take(4 * r * m.p);                // sup_val
  o[10] = L.take(16 * r * ((m.n + 255) / 256));   // partials
  o[11] = L.take(4 * (size_t)m.ldU);         // y_out
  o[12] = L.take(4 * (size_t)m.ldX);         // x_out
  o[13] = L.take(8 * (size_t)m.p);           // support_out
  o[14] = L.take(4 * r * 5);                 // status, iters, nnz, act, rank
  o[15] = L.take(8 * r * 6);                 // F, F_prev, gamma, f, ev (+ pad)
  o[16] = L.take(4 * r * 3);                 // thr, tprev, xfast
  o[17] = L.take(sizeof(Ctrl) * 2);          // ctrl of each parity
  o[18] = L.take(16);                        // best, nnz_out
  o[19] = L.take(sizeof(CUtensorMap) * 4);   // maps
  return L.off;
}

// admit one problem: its block, its starts normalised, its first active list (for sweep k + 1)
int admit_one(spca_group *g, const spca_problem &q, int tag) {
  cudaStream_t st = g->stream;
  Member m;
  m.h = q.h;
  m.P = q.prm;
  m.res = q.res;
  m.tag = tag;
  m.r = m.P.r;
  m.n = (int)m.h->n;
  m.p = (int)m.h->p;
  m.target = is_pen(m.P.form) && m.P.gamma_mode == SPCA_GAMMA_TARGET_NNZ;
  m.ldX = pad_ld(m.p);
  m.ldU = pad_ld(m.n);
  size_t o[20];
  const size_t bytes = member_layout(m, o);
  GCK(cudaMallocFromPoolAsync((void **)&m.mem, bytes, g->mempool, st));
  auto at = [&](int i) { return m.mem + o[i]; };
  GCK(cudaMemsetAsync(m.mem, 0, o[5], st));
  GProb &d = m.d;
  d.n = m.n;
  d.p = m.p;
  d.r = m.r;
  d.form = m.P.form;
  d.ldX = m.ldX;
  d.ldU = m.ldU;
  d.ldAT = m.h->ldAT;
  d.AT32 = m.h->AT32;
  d.AT16 = m.h->resident16 ? static_cast<const __half *>(m.h->ATpl) : nullptr;
  d.at_inv = m.h->at_inv;
  d.X = reinterpret_cast<float *>(at(0));
  d.V = nullptr;      // set with the pools (build_tables)
  d.U = reinterpret_cast<float *>(at(2));
  d.Xpl = reinterpret_cast<__half *>(at(3));
  d.Ypl = nullptr;
  d.xps = (int64_t)m.r * m.ldX;
  d.yps = 0;
  d.x_scale = reinterpret_cast<float *>(at(6));
  d.x_inv = reinterpret_cast<float *>(at(7));
  d.sup_idx = reinterpret_cast<int *>(at(8));
  d.sup_val = reinterpret_cast<float *>(at(9));
  m.partials = reinterpret_cast<double *>(at(10));
  m.y_out = reinterpret_cast<float *>(at(11));
  m.x_out = reinterpret_cast<float *>(at(12));
  m.support_out = reinterpret_cast<int64_t *>(at(13));
  int *ip = reinterpret_cast<int *>(at(14));
  double *dp = reinterpret_cast<double *>(at(15));
  float *fp = reinterpret_cast<float *>(at(16));
  StartState &s = d.st;
  s.status = ip;
  s.iters = ip + m.r;
  s.nnz = ip + 2 * m.r;
  d.act = ip + 3 * m.r;
  d.rank = ip + 4 * m.r;
  s.F = dp;
  s.F_prev = dp + m.r;
  s.gamma = dp + 2 * m.r;
  s.f = dp + 3 * m.r;
  s.ev = dp + 4 * m.r;
  s.thr = fp;
  s.tprev = fp + m.r;
  s.xfast = reinterpret_cast<int *>(fp + 2 * m.r);
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(at(17));
  d.ctrl[0] = ctrl;
  d.ctrl[1] = ctrl + 1;
  m.best = reinterpret_cast<int *>(at(18));
  m.nnz_out = reinterpret_cast<int64_t *>(at(18) + 8);
  m.maps = reinterpret_cast<CUtensorMap *>(at(19));
  GCK(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl) * 2, st));
  XstepArgs &a = d.xa;
  a = XstepArgs{};
  a.form = m.P.form;
  a.p = m.p;
  a.s = m.P.s;
  a.thr_fixed = uses_U(m.P.form) ? u_threshold(m.P.gamma) : (float)m.P.gamma;
  a.gamma_fixed = m.P.gamma;
  a.tol = m.P.tol;
  a.max_iter = m.P.max_iter;
  a.cap = m.p;
  a.sparse_cap = m.p;   // the support gather serves every support after the first sweep
  a.schedule = 1;
  a.target = m.target;
  a.calib_sweeps = m.target ? m.P.gamma_calib_sweeps : 0;
  a.lowp_sweeps = 0;
  a.stop_enabled = m.P.tol >= 0.0 ? 1 : 0;
  d.gamma0 = is_pen(m.P.form) && !m.target ? m.P.gamma : 0.0;
  d.ld0 = m.ldX;
  d.key = seed_key(m.P.seed);
  d.x0 = nullptr;
  if (q.x0) {   // the given starts, copied into X and normalised there (they must be finite)
    d.x0 = d.X;
    GCK(cudaMemcpy2DAsync(d.X, m.ldX * sizeof(float), q.x0, (size_t)m.p * sizeof(float), (size_t)m.p * sizeof(float),
                          m.r, m.P.x0_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    // the caller reads the error word once for all the problems of its call
    GCK(launch_check_finite(d.X, m.r, m.p, m.ldX, g->d_err, st));
  }
  CUtensorMap maps[3];
  maps[0] = m.h->pmA.m[0];
  maps[1] = m.h->pmAT.m[0];
  GCK(make_plane_map(&maps[2], d.Xpl, m.r, m.ldX, 2, 64, 64));
  GCK(cudaMemcpyAsync(m.maps, maps, 3 * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
  // the starts (seeded, or x0 normalised) and the first active list are set up at the start of the
  // member's first sweep, in one launch each with every other member admitted for that sweep
  m.first_pending = true;
  g->members.push_back(m);
  g->tables_ok = false;
  return SPCA_OK;
}

// the tables of the current members: problem entries, start -> problem map, tile tasks (u for the
// members whose first sweep is pending, v for each parity), each task list ordered by falling K
int build_tables(spca_group *g) {
  const int np = (int)g->members.size();
  cudaStream_t st = g->stream;
  // pools: the members on one matrix whose v = A^T y takes the same plane products (two general
  // operands, y = +-1, or the leading planes of a resident 16-bit matrix) share one contraction,
  // their active starts side by side in one Y operand, so the matrix is read once per sweep for
  // all of them; member order within a pool is admission order
  struct PoolH {
    const void *mat;
    int type;
    std::vector<int> mem;
    int R = 0;
  };
  std::vector<PoolH> pools;
  std::vector<int> vbase(np), pool_of(np);
  for (int i = 0; i < np; ++i) {
    const Member &m = g->members[i];
    const int type = m.h->resident16 ? 2 : is_l1_var(m.P.form) ? 1 : 0;
    int q = 0;
    while (q < (int)pools.size() && !(pools[q].mat == m.h->shared && pools[q].type == type)) ++q;
    if (q == (int)pools.size()) {
      pools.emplace_back();
      pools[q].mat = m.h->shared;
      pools[q].type = type;
    }
    pool_of[i] = q;
    vbase[i] = pools[q].R;
    pools[q].R += m.r;
    pools[q].mem.push_back(i);
  }
  const int npool = (int)pools.size();
  bool lowp_all = true;
  for (const PoolH &q : pools) lowp_all = lowp_all && q.type == 2;
  g->lowp_all = lowp_all;
  if (g->tiles_auto) {   // the measured choices by start count (bench.py --tune), on the widest pool
    int widest = 0;
    for (const PoolH &q : pools) widest = std::max(widest, q.R);
    if (lowp_all) {   // one accumulator per tile: up to 256 columns, four stages
      g->bn = widest > 128 ? 256 : widest > 64 ? 128 : 64;
      g->stages = 4;
    } else {
      g->bn = widest > 64 ? 128 : 64;
      g->stages = widest > 64 ? 3 : 4;
    }
  }
  // the pools' V rows and Y planes: one block, zeroed when it is made (the planes' padded columns
  // stay zero: the y-step writes the first n of a row), kept while the pools' shapes are the same
  Layout PL;
  std::vector<size_t> oV(npool), oY(npool);
  std::vector<int64_t> sig;
  for (int q = 0; q < npool; ++q) {
    const Member &m0 = g->members[pools[q].mem[0]];
    oV[q] = PL.take(4 * (size_t)pools[q].R * m0.ldX);
    oY[q] = PL.take(2 * 2 * (size_t)pools[q].R * m0.ldU);
    sig.insert(sig.end(), {(int64_t)pools[q].R, m0.ldX, m0.ldU});
  }
  if (sig != g->pool_sig || !g->pool_mem) {
    if (g->pool_mem) GCK(cudaFreeAsync(g->pool_mem, st));
    g->pool_mem = nullptr;
    g->pool_sig.clear();
    GCK(cudaMallocFromPoolAsync((void **)&g->pool_mem, std::max<size_t>(PL.off, 256), g->mempool, st));
    GCK(cudaMemsetAsync(g->pool_mem, 0, std::max<size_t>(PL.off, 256), st));
    g->pool_sig = sig;
  }
  int R_all = 0;
  bool use_cand = false;
  for (const Member &m : g->members) {
    R_all += m.r;
    use_cand = use_cand || m.p >= kCandMinPGroup;
  }
  const size_t cand_row = sizeof(float) * kXstepCand + sizeof(int) * kXstepCand;
  if (use_cand && R_all > g->cand_cap) {
    const int cap = std::max(R_all, g->cand_cap + g->cand_cap / 2);
    if (g->cand_mem) GCK(cudaFreeAsync(g->cand_mem, st));
    g->cand_mem = nullptr;
    g->cand_cap = 0;
    GCK(cudaMallocFromPoolAsync((void **)&g->cand_mem, (cand_row + sizeof(int4)) * (size_t)cap, g->mempool, st));
    g->cand_cap = cap;
  }
  g->use_cand = use_cand;
  float *cand_val = use_cand ? reinterpret_cast<float *>(g->cand_mem) : nullptr;
  int *cand_idx = use_cand ? reinterpret_cast<int *>(g->cand_mem + sizeof(float) * kXstepCand * (size_t)g->cand_cap)
                           : nullptr;
  int4 *cand_meta = use_cand ? reinterpret_cast<int4 *>(g->cand_mem + cand_row * (size_t)g->cand_cap) : nullptr;
  int R = 0, max_n = 1, max_p = 1, max_p_small = 0;
  bool any_large_p = false;
  for (int i = 0; i < np; ++i) {
    Member &m = g->members[i];
    const int q = pool_of[i];
    m.d.cand_val = use_cand ? cand_val + (int64_t)R * kXstepCand : nullptr;
    m.d.cand_idx = use_cand ? cand_idx + (int64_t)R * kXstepCand : nullptr;
    m.d.meta = use_cand ? cand_meta + R : nullptr;
    m.d.start0 = R;
    m.d.first = m.first_pending ? 1 : 0;
    m.d.vbase = vbase[i];
    m.d.V = reinterpret_cast<float *>(g->pool_mem + oV[q]) + (int64_t)vbase[i] * m.ldX;
    m.d.Ypl = reinterpret_cast<__half *>(g->pool_mem + oY[q]);
    m.d.yps = (int64_t)pools[q].R * m.ldU;
    R += m.r;
    max_n = std::max(max_n, m.n);
    max_p = std::max(max_p, m.p);
    if (m.p <= kXstepSmemMaxP)
      max_p_small = std::max(max_p_small, m.p);
    else
      any_large_p = true;
  }
  // the device tables: problems, start -> problem, tasks (u of the pending members; v of the
  // pools, one copy per parity), active counts, tile lists, pools, pool members, pool counts,
  // column maps, Y row offsets, the pools' Y plane maps
  Layout L;
  const size_t oP = L.take(sizeof(GProb) * np), oS = L.take(sizeof(int) * R),
               oT = L.take(sizeof(GTask) * (np + 2 * npool)), oA = L.take(sizeof(int) * np);
  std::vector<int2> tl[3];
  const size_t oPool = L.take(sizeof(GPool) * npool), oPM = L.take(sizeof(int) * np),
               oPC = L.take(sizeof(int) * npool), oCM = L.take(sizeof(int) * R), oYO = L.take(sizeof(int) * np),
               oMap = L.take(sizeof(CUtensorMap) * npool);
  // (the tile lists go last: their sizes are known once the tasks are)
  std::vector<int> start_prob(R);
  for (int i = 0; i < np; ++i)
    for (int c = 0; c < g->members[i].r; ++c) start_prob[g->members[i].d.start0 + c] = i;
  std::vector<GProb> P(np);
  for (int i = 0; i < np; ++i) P[i] = g->members[i].d;
  std::vector<GTask> tasks(np + 2 * npool);
  // the tile list of a set of tasks: by falling K, and the tasks on one matrix walked together by
  // M tile (their tiles of a row tile side by side: they read the same A tile)
  auto tiles_of = [&](GTask *base, std::vector<GTask> &T, std::vector<const void *> &mat, std::vector<int2> &tiles) {
    std::vector<int> order(T.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      if (T[a].kblocks != T[b].kblocks) return T[a].kblocks > T[b].kblocks;
      return reinterpret_cast<uintptr_t>(mat[a]) < reinterpret_cast<uintptr_t>(mat[b]);
    });
    for (size_t k = 0; k < order.size(); ++k) base[k] = T[order[k]];
    tiles.clear();
    for (size_t a = 0; a < order.size();) {
      size_t b = a + 1;
      while (b < order.size() && mat[order[b]] == mat[order[a]] && base[b].mt == base[a].mt) ++b;
      for (int tm = 0; tm < base[a].mt; ++tm)
        for (size_t k = a; k < b; ++k)
          for (int tn = 0; tn < base[k].nt; ++tn) tiles.push_back(make_int2((int)k, tm * base[k].nt + tn));
      a = b;
    }
    return (int)tiles.size();
  };
  // u = A x of the members whose first sweep is pending (it reads parity k & 1)
  int n_u = 0;
  {
    std::vector<GTask> T;
    std::vector<const void *> mat;
    for (int i = 0; i < np; ++i) {
      const Member &m = g->members[i];
      if (!m.first_pending) continue;
      const bool lowp = m.h->resident16;   // its A has the leading plane only
      GTask t{};
      t.pmap = m.maps + 0;
      t.qmap = m.maps + 2;
      t.M = m.n;
      t.kblocks = (m.p + 63) / 64;
      t.nmax = m.r;
      t.na = lowp ? 1 : 2;
      t.nb = lowp ? 1 : 2;
      t.n_dev = &m.d.ctrl[g->k & 1]->active;
      t.col_map = m.d.act;
      t.out = m.d.U;
      t.ldo = m.ldU;
      t.row_inv = m.h->a_inv;
      t.col_inv = m.d.x_inv;
      t.q_inv = 1.0f;
      t.pairs = lowp ? pairs_hi() : pairs_general();
      t.mt = (t.M + TC_BM_ROWS - 1) / TC_BM_ROWS;
      t.nt = (m.r + g->bn - 1) / g->bn;
      T.push_back(t);
      mat.push_back(m.h->shared);
    }
    n_u = (int)T.size();
    g->total_u = tiles_of(tasks.data(), T, mat, tl[0]);
  }
  // v = A^T y of the pools (one task each; the pool kernel fills the counts and column maps of the
  // sweep's parity, so both parities take the same tasks)
  {
    std::vector<GTask> T;
    std::vector<const void *> mat;
    int64_t cm = 0;
    for (int q = 0; q < npool; ++q) {
      const Member &m0 = g->members[pools[q].mem[0]];
      const int type = pools[q].type;
      GTask t{};
      t.pmap = m0.maps + 1;
      t.qmap = reinterpret_cast<const CUtensorMap *>(g->tab + oMap) + q;
      t.M = m0.p;
      t.kblocks = (m0.n + 63) / 64;
      t.nmax = pools[q].R;
      t.na = type == 2 ? 1 : 2;
      t.nb = type == 0 ? 2 : 1;
      t.n_dev = reinterpret_cast<int *>(g->tab + oPC) + q;
      t.col_map = reinterpret_cast<int *>(g->tab + oCM) + cm;
      t.out = reinterpret_cast<float *>(g->pool_mem + oV[q]);
      t.ldo = m0.ldX;
      t.row_inv = m0.h->at_inv;
      t.col_inv = nullptr;
      t.q_inv = kQInv;
      t.pairs = type == 2 ? pairs_hi() : type == 1 ? pairs_sign() : pairs_general();
      t.mt = (t.M + TC_BM_ROWS - 1) / TC_BM_ROWS;
      t.nt = (pools[q].R + g->bn - 1) / g->bn;
      T.push_back(t);
      mat.push_back(pools[q].mat);
      cm += pools[q].R;
    }
    g->total_v = tiles_of(tasks.data() + np, T, mat, tl[1]);
    for (int q = 0; q < npool; ++q) tasks[np + npool + q] = tasks[np + q];
    tl[2] = tl[1];
  }
  const size_t oL0 = L.take(sizeof(int2) * tl[0].size()), oL1 = L.take(sizeof(int2) * tl[1].size());
  if (L.off > g->tab_bytes) {
    // (the tasks hold addresses inside the table: a new table means new tasks, built again)
    GCK(cudaStreamSynchronize(st));
    if (g->tab) cudaFree(g->tab);
    g->tab = nullptr;
    g->tab_bytes = 0;
    GCK(cudaMalloc((void **)&g->tab, L.off + (L.off >> 2)));
    g->tab_bytes = L.off + (L.off >> 2);
    for (GroupGraph &q : g->graphs)
      if (q.exec) cudaGraphExecDestroy(q.exec);
    g->graphs.clear();
    return build_tables(g);
  }
  if (g->h_active_cap < np) {
    if (g->h_active) cudaFreeHost(g->h_active);
    g->h_active = nullptr;
    g->h_active_cap = 0;
    GCK(cudaMallocHost((void **)&g->h_active, sizeof(int) * np));
    g->h_active_cap = np;
  }
  char *tab = g->tab;
  g->dP = reinterpret_cast<GProb *>(tab + oP);
  g->d_start_prob = reinterpret_cast<int *>(tab + oS);
  g->d_tasks = reinterpret_cast<GTask *>(tab + oT);
  g->d_active = reinterpret_cast<int *>(tab + oA);
  g->d_tiles[0] = reinterpret_cast<int2 *>(tab + oL0);
  g->d_tiles[1] = g->d_tiles[2] = reinterpret_cast<int2 *>(tab + oL1);
  g->d_pools = reinterpret_cast<GPool *>(tab + oPool);
  g->d_pool_members = reinterpret_cast<int *>(tab + oPM);
  g->npool = npool;
  // pools, their member lists and the members' Y row offset words
  std::vector<GPool> GP(npool);
  std::vector<int> pm;
  int64_t cm = 0;
  for (int q = 0; q < npool; ++q) {
    GP[q].first = (int)pm.size();
    GP[q].nmem = (int)pools[q].mem.size();
    GP[q].count = reinterpret_cast<int *>(tab + oPC) + q;
    GP[q].colmap = reinterpret_cast<int *>(tab + oCM) + cm;
    pm.insert(pm.end(), pools[q].mem.begin(), pools[q].mem.end());
    cm += pools[q].R;
  }
  for (int i = 0; i < np; ++i) {
    P[i].yoff = reinterpret_cast<int *>(tab + oYO) + i;
    g->members[i].d.yoff = P[i].yoff;
  }
  std::vector<CUtensorMap> maps(npool);
  for (int q = 0; q < npool; ++q)
    GCK(make_plane_map(&maps[q], g->pool_mem + oY[q], pools[q].R, g->members[pools[q].mem[0]].ldU, 2, 64, 64));
  // (pageable sources: each copy returns once its data are staged, so the vectors may go)
  GCK(cudaMemcpyAsync(g->dP, P.data(), sizeof(GProb) * np, cudaMemcpyHostToDevice, st));
  GCK(cudaMemcpyAsync(g->d_start_prob, start_prob.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
  GCK(cudaMemcpyAsync(g->d_tasks, tasks.data(), sizeof(GTask) * tasks.size(), cudaMemcpyHostToDevice, st));
  if (!tl[0].empty())
    GCK(cudaMemcpyAsync(g->d_tiles[0], tl[0].data(), sizeof(int2) * tl[0].size(), cudaMemcpyHostToDevice, st));
  if (!tl[1].empty())
    GCK(cudaMemcpyAsync(g->d_tiles[1], tl[1].data(), sizeof(int2) * tl[1].size(), cudaMemcpyHostToDevice, st));
  GCK(cudaMemcpyAsync(g->d_pools, GP.data(), sizeof(GPool) * npool, cudaMemcpyHostToDevice, st));
  GCK(cudaMemcpyAsync(g->d_pool_members, pm.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st));
  GCK(cudaMemcpyAsync(tab + oMap, maps.data(), sizeof(CUtensorMap) * npool, cudaMemcpyHostToDevice, st));
  g->R = R;
  g->n_u = n_u;
  g->max_n = max_n;
  g->max_p = max_p;
  g->max_p_small = max_p_small;
  g->any_large_p = any_large_p;
  g->tables_ok = true;
  return SPCA_OK;
}

// the launches of global sweep k (the members' tables as built)
cudaError_t enqueue_sweep(spca_group *g, int64_t k, bool first_of_segment) {
  cudaStream_t st = g->stream;
  const int np = (int)g->members.size();
  const int cur = (int)((k - 1) & 1), nxt = (int)(k & 1);
  const uint64_t wait_ns = 2000000000ull;
  cudaError_t e = cudaSuccess;
  if (first_of_segment && g->n_u > 0) {
    // the first sweep of the members admitted before this segment: their starts and active lists
    // (parity cur: the control words this sweep reads), then the dense u = A x
    e = launch_g_start_init(g->dP, g->d_start_prob, g->R, st);
    if (e == cudaSuccess) e = launch_g_active(g->dP, np, cur, true, st);
    if (e == cudaSuccess) e = launch_g_xplanes(g->dP, g->d_start_prob, g->R, st);
    if (e == cudaSuccess)
      e = launch_gemm_grouped(g->d_tasks, g->d_tiles[0], g->total_u, g->bn, g->stages, g->lowp_all, g->sms, g->d_err,
                              wait_ns, st);
  }
  // the pools' Y rows, counts and column maps for this sweep's active lists
  if (e == cudaSuccess) e = launch_g_pools(g->d_pools, g->npool, g->dP, g->d_pool_members, cur, st);
  if (e == cudaSuccess) e = launch_g_gather(g->dP, g->d_start_prob, g->R, g->max_n, st);
  if (e == cudaSuccess) e = launch_g_ystep(g->dP, g->d_start_prob, g->R, st);
  if (e == cudaSuccess)
    e = launch_gemm_grouped(g->d_tasks + np + cur * g->npool, g->d_tiles[1 + cur], g->total_v, g->bn, g->stages,
                            g->lowp_all, g->sms, g->d_err, wait_ns, st);
  if (e == cudaSuccess) e = launch_g_ctrl(g->dP, np, nxt, 1, nullptr, st);
  if (e == cudaSuccess)
    e = launch_g_xstep(g->dP, g->d_start_prob, g->R, g->max_p_small, g->any_large_p, g->use_cand, nxt, g->sms, st);
  if (e == cudaSuccess) e = launch_g_active(g->dP, np, nxt, false, st);
  return e;
}

// Table 1 objective of every start, the best start and its outputs for the listed members, then
// their results to the host: every piece gathered into one staging buffer by one launch, one copy
// to pinned host memory, one synchronisation
int finish_members(spca_group *g, const std::vector<Member *> &list) {
  if (list.empty()) return SPCA_OK;
  cudaStream_t st = g->stream;
  struct Piece {
    size_t off;
    int64_t bytes;
  };
  std::vector<CopyDesc> desc;
  std::vector<std::vector<Piece>> pieces(list.size());
  size_t off = 0;
  auto add = [&](size_t k, const void *src, int64_t bytes) {
    desc.push_back(CopyDesc{src, nullptr, bytes});
    pieces[k].push_back(Piece{off, bytes});
    off += (bytes + 15) / 16 * 16;
  };
  for (size_t k = 0; k < list.size(); ++k) {
    Member &m = *list[k];
    const GProb &d = m.d;
    if (m.h->resident16)
      GCK(launch_finalise_h(m.P.form, d.AT16, d.at_inv, m.h->ldAT, m.n, d.st, m.r, d.U, m.ldU, d.sup_idx, d.sup_val,
                            m.p, m.partials, st));
    else
      GCK(launch_finalise(m.P.form, m.h->AT32, m.h->ldAT, m.n, m.p, d.X, m.ldX, d.st, m.r, d.U, m.ldU, d.sup_idx,
                          d.sup_val, m.p, m.partials, st));
    GCK(launch_best(m.P.form, m.target, d.st, m.r, m.best, st));
    GCK(launch_best_outputs(m.P.form, m.best, d.U, m.ldU, m.n, d.X, m.ldX, m.p, m.y_out, m.x_out, m.support_out,
                            m.nnz_out, st));
    const int64_t r = m.r;
    add(k, d.st.status, 4 * r);
    add(k, d.st.iters, 4 * r);
    add(k, d.st.f, 8 * r);
    add(k, d.st.ev, 8 * r);
    add(k, d.st.gamma, 8 * r);
    add(k, d.st.F, 8 * r);
    add(k, m.best, 4);
    add(k, m.nnz_out, 8);
    add(k, m.x_out, 4 * (int64_t)m.p);
    add(k, m.y_out, 4 * (int64_t)m.n);
    add(k, m.support_out, 8 * (int64_t)m.p);
  }
  if (off > g->stage_bytes) {
    GCK(cudaStreamSynchronize(st));
    if (g->stage_d) cudaFree(g->stage_d);
    if (g->stage_h) cudaFreeHost(g->stage_h);
    g->stage_d = nullptr;
    g->stage_h = nullptr;
    g->stage_bytes = 0;
    GCK(cudaMalloc((void **)&g->stage_d, off));
    GCK(cudaMallocHost((void **)&g->stage_h, off));
    g->stage_bytes = off;
  }
  const size_t dbytes = sizeof(CopyDesc) * desc.size();
  if (dbytes > g->desc_bytes) {
    GCK(cudaStreamSynchronize(st));
    if (g->desc_d) cudaFree(g->desc_d);
    g->desc_d = nullptr;
    g->desc_bytes = 0;
    GCK(cudaMalloc((void **)&g->desc_d, dbytes));
    g->desc_bytes = dbytes;
  }
  size_t q = 0;
  for (size_t k = 0; k < list.size(); ++k)
    for (const Piece &pc : pieces[k]) desc[q++].dst = g->stage_d + pc.off;
  GCK(cudaMemcpyAsync(g->desc_d, desc.data(), dbytes, cudaMemcpyHostToDevice, st));
  GCK(launch_copy_list(g->desc_d, (int)desc.size(), st));
  GCK(cudaMemcpyAsync(g->stage_h, g->stage_d, off, cudaMemcpyDeviceToHost, st));
  GCK(cudaStreamSynchronize(st));
  for (size_t k = 0; k < list.size(); ++k) {
    Member &m = *list[k];
    const int r = m.r;
    const std::vector<Piece> &pc = pieces[k];
    const char *H = g->stage_h;
    const int *status = reinterpret_cast<const int *>(H + pc[0].off);
    const int *iters = reinterpret_cast<const int *>(H + pc[1].off);
    const double *f = reinterpret_cast<const double *>(H + pc[2].off);
    const double *ev = reinterpret_cast<const double *>(H + pc[3].off);
    const double *gam = reinterpret_cast<const double *>(H + pc[4].off);
    const double *F = reinterpret_cast<const double *>(H + pc[5].off);
    const int best = *reinterpret_cast<const int *>(H + pc[6].off);
    const int64_t nnz = *reinterpret_cast<const int64_t *>(H + pc[7].off);
    spca_result *res = m.res;
    if (res->x) memcpy(res->x, H + pc[8].off, (size_t)m.p * 4);
    if (res->y) memcpy(res->y, H + pc[9].off, (size_t)m.n * 4);
    if (res->support && nnz > 0) memcpy(res->support, H + pc[10].off, (size_t)nnz * 8);
    if (res->start_x)
      GCK(cudaMemcpy2DAsync(res->start_x, (size_t)m.p * 4, m.d.X, m.ldX * 4, (size_t)m.p * 4, r,
                            cudaMemcpyDeviceToHost, st));
    int64_t sweeps = 0;
    int nconv = 0, ndeg = 0;
    for (int c = 0; c < r; ++c) {
      sweeps += iters[c];
      nconv += status[c] == SPCA_ST_CONVERGED;
      ndeg += status[c] == SPCA_ST_DEGENERATE;
    }
    const bool pen = is_pen(m.P.form);
    res->objective = f[best];
    res->explained_variance = ev[best];
    res->gamma = pen ? gam[best] : 0.0;
    res->best_start = best;
    res->best_iters = iters[best];
    res->best_status = status[best];
    res->converged = nconv;
    res->degenerate = ndeg;
    res->sweeps_total = sweeps;
    res->nnz = nnz;
    for (int c = 0; c < r; ++c) {
      if (res->start_objective) res->start_objective[c] = f[c];
      if (res->start_explained) res->start_explained[c] = ev[c];
      if (res->start_F) res->start_F[c] = F[c];
      if (res->start_iters) res->start_iters[c] = iters[c];
      if (res->start_status) res->start_status[c] = status[c];
      if (res->start_gamma) res->start_gamma[c] = pen ? gam[c] : 0.0;
    }
  }
  GCK(cudaStreamSynchronize(st));   // the start_x copies
  return SPCA_OK;
}

void release_member(spca_group *g, Member &m) {
  if (m.mem) cudaFreeAsync(m.mem, g->stream);
  m.mem = nullptr;
}

// run `sweeps` sweeps for the current members (captured into a graph when `capture`), then the
// active counts; finished members (no active start) are finalised and retired when `retire`
int run_segment(spca_group *g, int sweeps, bool capture, bool retire, int *finished, int cap, int *nfin) {
  cudaStream_t st = g->stream;
  if (nfin) *nfin = 0;
  if (g->members.empty()) return SPCA_OK;
  if (!g->tables_ok) GRC(build_tables(g));
  const int np = (int)g->members.size();
  if (capture) {
    uint64_t key = 1469598103934665603ull;
    key = fnv(key, &g->tab, sizeof g->tab);
    for (const Member &m : g->members) key = fnv(key, &m.d, sizeof m.d);
    const int64_t par = g->k & 1;
    const int pend = g->n_u;
    key = fnv(key, &par, sizeof par);
    key = fnv(key, &pend, sizeof pend);
    key = fnv(key, &sweeps, sizeof sweeps);
    key = fnv(key, &g->bn, sizeof g->bn);
    key = fnv(key, &g->lowp_all, sizeof g->lowp_all);
    key = fnv(key, &g->stages, sizeof g->stages);
    GroupGraph *gg = nullptr;
    for (GroupGraph &q : g->graphs)
      if (q.key == key) gg = &q;
    if (!gg) {
      if (g->graphs.size() > 32) {
        GCK(cudaStreamSynchronize(st));
        for (GroupGraph &q : g->graphs)
          if (q.exec) cudaGraphExecDestroy(q.exec);
        g->graphs.clear();
      }
      g->graphs.emplace_back();
      gg = &g->graphs.back();
      gg->key = key;
      cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
      cudaError_t be = cudaSuccess;
      if (ce == cudaSuccess) {
        for (int j = 0; j < sweeps && be == cudaSuccess; ++j) be = enqueue_sweep(g, g->k + 1 + j, j == 0);
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
  } else {
    for (int j = 0; j < sweeps; ++j) GCK(enqueue_sweep(g, g->k + 1 + j, j == 0));
  }
  g->k += sweeps;
  if (g->n_u > 0) {   // the pending members have had their first sweep
    for (Member &m : g->members) m.first_pending = false;
    g->tables_ok = false;
  }
  GCK(launch_g_ctrl(g->dP, np, (int)(g->k & 1), 0, g->d_active, st));
  GCK(cudaMemcpyAsync(g->h_active, g->d_active, sizeof(int) * np, cudaMemcpyDeviceToHost, st));
  GCK(cudaMemcpyAsync(g->h_err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GCK(cudaStreamSynchronize(st));
  if (*g->h_err) {
    const int code = *g->h_err;
    cudaMemsetAsync(g->d_err, 0, sizeof(int), st);
    return gfail(g, code, "a device-side wait timed out");
  }
  if (!retire) return SPCA_OK;
  std::vector<Member> keep;
  std::vector<Member *> done;
  int nf = 0;
  const std::vector<int> active(g->h_active, g->h_active + np);
  for (int i = 0; i < np; ++i) {
    Member &m = g->members[i];
    if (active[i] > 0) continue;
    done.push_back(&m);
    if (finished && nf < cap) finished[nf] = m.tag;
    ++nf;
  }
  GRC(finish_members(g, done));
  for (int i = 0; i < np; ++i) {
    Member &m = g->members[i];
    if (active[i] > 0) keep.push_back(m);
    else release_member(g, m);
  }
  if (nf > 0) {
    g->members.swap(keep);
    g->tables_ok = false;
  }
  if (nfin) *nfin = nf;
  return SPCA_OK;
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
      cudaMallocHost((void **)&g->h_err, sizeof(int)) != cudaSuccess ||
      cudaMalloc((void **)&g->d_err, sizeof(int)) != cudaSuccess ||
      cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream) != cudaSuccess) {
    spca_group_destroy(g);
    return SPCA_E_CUDA;
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  uint64_t keep = ~0ull;
  if (cudaMemPoolCreate(&g->mempool, &props) != cudaSuccess ||
      cudaMemPoolSetAttribute(g->mempool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
    spca_group_destroy(g);
    return SPCA_E_CUDA;
  }
  *out = g;
  return SPCA_OK;
}

void spca_group_destroy(spca_group *g) {
  if (!g) return;
  for (Member &m : g->members) release_member(g, m);
  g->members.clear();
  if (g->pool_mem && g->stream) cudaFreeAsync(g->pool_mem, g->stream);
  if (g->cand_mem && g->stream) cudaFreeAsync(g->cand_mem, g->stream);
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (GroupGraph &q : g->graphs)
    if (q.exec) cudaGraphExecDestroy(q.exec);
  if (g->tab) cudaFree(g->tab);
  if (g->stage_d) cudaFree(g->stage_d);
  if (g->stage_h) cudaFreeHost(g->stage_h);
  if (g->desc_d) cudaFree(g->desc_d);
  if (g->d_err) cudaFree(g->d_err);
  if (g->h_active) cudaFreeHost(g->h_active);
  if (g->h_err) cudaFreeHost(g->h_err);
  if (g->order_ev) cudaEventDestroy(g->order_ev);
  if (g->stream) cudaStreamDestroy(g->stream);
  if (g->mempool) cudaMemPoolDestroy(g->mempool);   // (every block was freed and the stream drained)
  delete g;
}

const char *spca_group_last_error(const spca_group *g) { return g ? g->last_error : ""; }

int spca_group_set_tiles(spca_group *g, const spca_group_tiles *tiles) {
  if (!g) return SPCA_E_INVALID;
  if (!tiles || (!tiles->tile_n && !tiles->stages)) {   // chosen with the tables
    if (!g->tiles_auto) g->tables_ok = false;
    g->tiles_auto = true;
    return SPCA_OK;
  }
  const int bn = tiles->tile_n, stages = tiles->stages;
  if (!grouped_config_ok(bn, stages, false)) return gfail(g, SPCA_E_INVALID, "unknown tile shape (tile_n, stages)");
  if (bn != g->bn || g->tiles_auto) g->tables_ok = false;   // the N tiles of the tasks change
  g->tiles_auto = false;
  g->bn = bn;
  g->stages = stages;
  return SPCA_OK;
}

int spca_group_admit(spca_group *g, spca_problem *probs, int count, const int *tags) {
  if (!g || (count > 0 && !probs) || count < 0) return gfail(g, SPCA_E_INVALID, "NULL group or problems");
  if ((int64_t)g->members.size() + count > kGroupMaxTasks)
    return gfail(g, SPCA_E_UNSUPPORTED, "more than 1024 problems in one group");
  for (int i = 0; i < count; ++i)
    if (const char *bad = check_problem(probs[i])) return gfail(g, SPCA_E_INVALID, bad);
  GCK(cudaEventRecord(g->order_ev, g->user));
  GCK(cudaStreamWaitEvent(g->stream, g->order_ev, 0));
  const size_t before = g->members.size();
  auto undo = [&](int rc) {   // none of this call's problems stays admitted
    for (size_t j = before; j < g->members.size(); ++j) release_member(g, g->members[j]);
    g->members.resize(before);
    g->tables_ok = false;
    return rc;
  };
  bool given = false;
  for (int i = 0; i < count; ++i) given = given || probs[i].x0;
  // no grouped launch is in flight between segments, so the error word is free for the x0 checks
  if (given && cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream) != cudaSuccess)
    return gfail(g, SPCA_E_CUDA, "cudaMemsetAsync failed");
  for (int i = 0; i < count; ++i) {
    const int rc = admit_one(g, probs[i], tags ? tags[i] : i);
    if (rc != SPCA_OK) return undo(rc);
  }
  if (given) {   // one synchronisation for every given start of the call
    if (cudaMemcpyAsync(g->h_err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
        cudaStreamSynchronize(g->stream) != cudaSuccess)
      return undo(gfail(g, SPCA_E_CUDA, "reading the x0 check failed"));
    if (*g->h_err) {
      cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream);
      return undo(gfail(g, SPCA_E_INVALID, "x0 has a non-finite entry"));
    }
  }
  return SPCA_OK;
}

int spca_group_step(spca_group *g, int sweeps, int *finished, int cap, int *nfinished) {
  if (!g || sweeps < 1 || (cap > 0 && !finished)) return gfail(g, SPCA_E_INVALID, "bad arguments");
  GCK(cudaEventRecord(g->order_ev, g->user));
  GCK(cudaStreamWaitEvent(g->stream, g->order_ev, 0));
  return run_segment(g, sweeps, false, true, finished, cap, nfinished);
}

int spca_group_pending(const spca_group *g) { return g ? (int)g->members.size() : 0; }

int spca_solve_group(spca_group *g, spca_problem *probs, int count, const spca_group_tiles *tiles) {
  if (!g || !probs || count < 1) return gfail(g, SPCA_E_INVALID, "NULL group or problems, or count < 1");
  if (!g->members.empty()) return gfail(g, SPCA_E_BUSY, "the group has admitted problems in progress");
  GRC(spca_group_set_tiles(g, tiles));
  GRC(spca_group_admit(g, probs, count, nullptr));
  // every member stays in the tables until the last one is done, so every segment but the first
  // (which holds the members' first sweeps) replays one captured graph
  int max_iter = 1;
  for (const Member &m : g->members) max_iter = std::max(max_iter, m.P.max_iter);
  const int check_every = 4;
  int rc = SPCA_OK;
  for (int64_t done = 0; done < max_iter && rc == SPCA_OK;) {
    const int seg = (int)std::min<int64_t>(check_every, max_iter - done);
    rc = run_segment(g, seg, true, false, nullptr, 0, nullptr);
    done += seg;
    if (rc != SPCA_OK) break;
    int64_t active = 0;
    for (size_t i = 0; i < g->members.size(); ++i) active += g->h_active[i];
    if (active == 0) break;
  }
  if (rc == SPCA_OK) {
    std::vector<Member *> all;
    for (Member &m : g->members) all.push_back(&m);
    rc = finish_members(g, all);
  }
  for (Member &m : g->members) release_member(g, m);
  g->members.clear();
  g->tables_ok = false;
  return rc;
}

}  // extern "C"
