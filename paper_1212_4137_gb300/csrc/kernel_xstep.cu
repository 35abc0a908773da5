// kernel_xstep.cu -- the x-step of Algorithm 2 for every active start (one CTA per start):
//   forms 1, 2   S3: T_s(v), the s largest |v_i| (ties: lower index), by radix select
//   forms 3, 4   S4: V_lambda(v) with lambda = lambda_s(v), by bisection on the sign of
//                    phi(lambda) = s ||V_lambda||_2^2 - ||V_lambda||_1^2, then the exact
//                    root of phi on the final piece (fixed active set)
//   forms 5, 6   S5: U_gamma(v), keep v_i^2 > gamma  (eq. 5)
//   forms 7, 8   S6: V_gamma(v), soft threshold       (eq. 6)
// then normalisation (Section 2.2), the Table 3 value F(x^(k+1), y^(k)), the stopping rule,
// and the support list (ascending indices) used by the sparse u = A x and the FP64 objective.
// Section 4.1's gamma rule (penalty forms) picks gamma so that exactly s entries survive.
//
// Layout: v is staged once in shared memory (p * 4 bytes up to XSTEP_SMEM_MAX, else read from
// global memory on every pass).  Each warp owns one contiguous index segment, so ordered work
// (support compaction, ranking of tied magnitudes) needs only warp ballots plus one scan over
// the 16 warps.  Reductions are in a fixed order: a start's result does not depend on the
// other starts or on scheduling.
#include <algorithm>
#include <cstdint>

#include "block_util.cuh"
#include "spca_internal.cuh"
#include "sweep_bodies.cuh"

namespace spca {

namespace {
constexpr int XT = 512;                        // threads per CTA
constexpr int XW = XT / 32;                    // warps per CTA
constexpr int XSTEP_SMEM_MAX = 200 * 1024;     // largest v staged in shared memory (bytes)
static_assert(kXstepSmemMaxP * 4 == XSTEP_SMEM_MAX, "the grouped x-step's split");

struct XShared {
  unsigned hist[256];
  double red_d[XW][2];
  float red_f[XW][2];
  int red_i[XW][2];
  int wcnt[XW];                                // per-warp counts of one pass
  int woff[XW];                                // their exclusive prefix over warps
  int digit, rem, cnt_bin;
  unsigned red_u[XW];
};

struct Seg {
  int lo, hi;
};
// this warp's index segment: 16 contiguous ranges, each a multiple of 32 long (the last shorter)
__device__ __forceinline__ Seg warp_seg(int p) {
  const int seg = (((p + XW - 1) / XW) + 31) / 32 * 32;
  const int w = threadIdx.x >> 5;
  Seg s;
  s.lo = min(p, w * seg);
  s.hi = min(p, s.lo + seg);
  return s;
}

// block sums of (f0, f1, i0, i1) in one round, FP32 in a fixed order; every thread gets them.
// (GB300's FP64 pipe is ~1/64 of FP32: FP64 stays out of the per-pass reductions.)
__device__ __forceinline__ void block_sum2f(float &f0, float &f1, int &i0, int &i1, XShared &sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  f0 = warp_sum_f(f0); f1 = warp_sum_f(f1); i0 = warp_sum_i(i0); i1 = warp_sum_i(i1);
  __syncthreads();
  if (lane == 0) { sh.red_f[w][0] = f0; sh.red_f[w][1] = f1; sh.red_i[w][0] = i0; sh.red_i[w][1] = i1; }
  __syncthreads();
  f0 = f1 = 0.0f; i0 = i1 = 0;
  for (int k = 0; k < XW; ++k) { f0 += sh.red_f[k][0]; f1 += sh.red_f[k][1]; i0 += sh.red_i[k][0]; i1 += sh.red_i[k][1]; }
}

// block sums of two FP64 values (each thread's value already accurate); the warp partials are
// combined by one thread, so the FP64 work is ~5 adds per thread
__device__ __forceinline__ void block_sum2d(double &d0, double &d1, XShared &sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  d0 = warp_sum_d(d0); d1 = warp_sum_d(d1);
  __syncthreads();
  if (lane == 0) { sh.red_d[w][0] = d0; sh.red_d[w][1] = d1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < XW; ++k) { a += sh.red_d[k][0]; b += sh.red_d[k][1]; }
    sh.red_d[0][0] = a; sh.red_d[0][1] = b;
  }
  __syncthreads();
  d0 = sh.red_d[0][0]; d1 = sh.red_d[0][1];
}

// compensated (Neumaier) FP32 accumulation: s + c carries the sum to ~2^-40 relative
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
  const float t = s + x;
  c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

// per-warp count -> exclusive offsets over warps (sh.woff) and the block total
__device__ __forceinline__ int warp_offsets(int my_warp_count, XShared &sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh.wcnt[w] = my_warp_count;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int k = 0; k < XW; ++k) { sh.woff[k] = acc; acc += sh.wcnt[k]; }
    sh.cnt_bin = acc;
  }
  __syncthreads();
  return sh.cnt_bin;
}

// The j-th largest (1 <= j <= p) of the keys |v_i| by MSB-first radix select over the digits
// bits 30..23 (the exponent), 22..15, 14..7, 6..0.  Histogram updates are aggregated per warp.
// If the chosen bin is exactly the remainder of the top j before the last digit, the search
// stops: every element of the bin is in the top j.  Then, with exact == false, *K is the bin's
// lower bound and *whole = true; with exact == true one more pass finds the bin's minimum,
// which is the j-th largest key.  Otherwise *need_eq / *eq_total describe ties at *K.
__device__ void radix_select(const float *vv, int p, int j, bool exact, XShared &sh, uint32_t *K,
                             bool *whole, int *need_eq, int *eq_total) {
  const int shifts[4] = {23, 15, 7, 0};
  const uint32_t wmask[4] = {0xFFu, 0xFFu, 0xFFu, 0x7Fu};
  const int lane = threadIdx.x & 31;
  const Seg sg = warp_seg(p);
  uint32_t prefix = 0u, mask = 0u;
  int rem = j;
  *whole = false;
  for (int t = 0; t < 4; ++t) {
    const int sh_ = shifts[t];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) sh.hist[b] = 0u;
    __syncthreads();
    for (int base = sg.lo; base < sg.hi; base += 32) {
      const int i = base + lane;
      const uint32_t key = (i < sg.hi) ? abs_key(vv[i]) : 0xFFFFFFFFu;
      const bool m = (i < sg.hi) && (key & mask) == prefix;
      const uint32_t bin = m ? (key >> sh_) & wmask[t] : 0xFFFFFFFFu;
      const unsigned peers = __match_any_sync(0xffffffffu, bin);
      if (m && lane == __ffs(peers) - 1) atomicAdd(&sh.hist[bin], (unsigned)__popc(peers));
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // warp 0 finds the bin holding the rem-th largest: lane l owns the bins
      // [top - l*per, top - l*per - per + 1] (descending), scans the lane sums from the top,
      // and the owning lane walks its own bins
      const int nb = (int)wmask[t] + 1, per = nb / 32, top = nb - 1 - lane * per;
      int lsum = 0;
      for (int q = 0; q < per; ++q) lsum += (int)sh.hist[top - q];
      int incl = lsum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int excl = incl - lsum;
      const bool mine = excl < rem && rem <= incl;
      const unsigned who = __ballot_sync(0xffffffffu, mine);
      if (mine && lane == __ffs(who) - 1) {
        int acc = excl, d = top;
        for (int q = 0; q < per - 1; ++q, --d) {
          if (acc + (int)sh.hist[d] >= rem) break;
          acc += (int)sh.hist[d];
        }
        sh.digit = d;
        sh.rem = rem - acc;
        sh.cnt_bin = (int)sh.hist[d];
      }
    }
    __syncthreads();
    prefix |= (uint32_t)sh.digit << sh_;
    mask |= wmask[t] << sh_;
    rem = sh.rem;
    const int cnt = sh.cnt_bin;
    __syncthreads();
    if (t == 3) {
      *K = prefix;
      *need_eq = rem;
      *eq_total = cnt;
      return;
    }
    if (cnt == rem) {  // the whole bin belongs to the top j
      if (!exact) {
        *K = prefix;
        *whole = true;
        return;
      }
      unsigned mn = 0xFFFFFFFFu;
      for (int base = sg.lo; base < sg.hi; base += 32) {
        const int i = base + lane;
        if (i < sg.hi) {
          const uint32_t key = abs_key(vv[i]);
          if ((key & mask) == prefix) mn = min(mn, key);
        }
      }
      // block minimum
      for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      if (lane == 0) sh.red_u[threadIdx.x >> 5] = mn;
      __syncthreads();
      unsigned m2 = 0xFFFFFFFFu;
      for (int k = 0; k < XW; ++k) m2 = min(m2, sh.red_u[k]);
      __syncthreads();
      *K = m2;
      *whole = true;
      return;
    }
  }
}

// lambda_s(v) (Section 2.1) when phi(0) < 0.  Bisection over the float keys of lambda in
// [lo0, max|v|] (phi(lo0) < 0 is known: lo0 = 0, or a lower bound checked by the caller) on
// the sign of phi, stopping as soon as no |v_i| lies strictly inside the bracket (the active
// set is then fixed); then the root of phi on that piece in FP64.
// *lo_out: the active set is {key_i > *lo_out}.
__device__ double lambda_s_bisect(const float *vv, int p, double s, uint32_t lo0, uint32_t maxkey, XShared &sh,
                                  uint32_t *lo_out) {
  const int lane = threadIdx.x & 31;
  const Seg sg = warp_seg(p);
  uint32_t lo = lo0, hi = maxkey;  // phi(key lo) < 0 <= phi(key hi)
  while (hi - lo > 1u) {
    const uint32_t mid = lo + (hi - lo) / 2u;
    const float lam = __uint_as_float(mid);
    float sw = 0.0f, sw2 = 0.0f;
    int in_lo = 0, in_hi = 0;  // elements strictly inside (lo, mid) and (mid, hi)
    for (int i = sg.lo + lane; i < sg.hi; i += 32) {
      const float a = fabsf(vv[i]);
      const uint32_t key = __float_as_uint(a);
      if (a > lam) {
        const float w = a - lam;
        sw += w;
        sw2 = fmaf(w, w, sw2);
      }
      in_lo += (key > lo && key < mid);
      in_hi += (key > mid && key < hi);
    }
    block_sum2f(sw, sw2, in_lo, in_hi, sh);
    const float phi = (float)s * sw2 - sw * sw;
    if (phi < 0.0f) {
      lo = mid;
      if (in_hi == 0) break;  // no magnitude strictly inside (mid, hi): active set fixed
    } else {
      hi = mid;
      if (in_lo == 0) break;
    }
  }
  // active set {key > lo}: k, S1, S2 (compensated per thread, FP64 across threads), then the
  // root of phi on this piece in FP64
  float a1 = 0.0f, c1 = 0.0f, a2 = 0.0f, c2 = 0.0f, fz = 0.0f;
  int kc = 0, unused = 0;
  for (int i = sg.lo + lane; i < sg.hi; i += 32) {
    const float a = fabsf(vv[i]);
    if (__float_as_uint(a) > lo) {
      ++kc;
      kahan_add(a1, c1, a);
      const float aa = a * a;
      kahan_add(a2, c2, aa);
      kahan_add(a2, c2, fmaf(a, a, -aa));   // exact square: aa + the FMA residual
    }
  }
  double s1 = (double)a1 + (double)c1, s2 = (double)a2 + (double)c2;
  block_sum2d(s1, s2, sh);
  block_sum2f(fz, fz, kc, unused, sh);
  const double k = (double)kc;
  const double flo = (double)__uint_as_float(lo), fhi = (double)__uint_as_float(hi);
  double lam;
  if (k <= s) {
    lam = flo;
  } else {
    double disc = s * (k * s2 - s1 * s1) / (k - s);
    if (disc < 0.0) disc = 0.0;
    lam = (s1 - sqrt(disc)) / k;
    lam = fmin(fmax(lam, flo), fhi);
  }
  *lo_out = lo;
  return lam;
}

// ---------------------------------------------------------------- the operator, then x
// mode 0: T_s with ties: keep key > K, plus the first need_eq of key == K in index order
// mode 1: hard threshold: keep key > tkey, value v            (U_gamma; T_s otherwise)
// mode 2: soft threshold: keep key > tkey, value sgn(v)(|v|-t)  (V_gamma, V_lambda)
struct XOp {
  int mode = 1;
  uint32_t K = 0u, tkey = 0u;
  int need_eq = 0;
  float tval = 0.0f;    // threshold value subtracted in mode 2
  double gam = 0.0;     // gamma in Table 1 units (penalties) or lambda_s (S4)
  float tnext = 0.0f;   // the threshold (|v| units) that seeds the next sweep's candidate filter
};

// Pass A (||w||_2^2 and nnz of the unnormalised result w), the Table 3 value, pass B (x = w /
// ||w||_2 and the support list in index order) and the per-start outputs, over vv[0 .. len):
// element i is entry map[i] of v and x (map == nullptr: entry i).
__device__ void xstep_finish(const XstepArgs &a, int c, const float *vv, int len, const int *map, const XOp &op,
                             float *x, StartState st, int *sup_idx, float *sup_val, Ctrl *ctrl, XShared &sh) {
  const int lane = threadIdx.x & 31;
  const int form = a.form;
  const Seg sg = warp_seg(len);

  // ---- ties (mode 0): offsets of each warp's equal keys in index order
  if (op.mode == 0) {
    int eq = 0;
    for (int i = sg.lo + lane; i < sg.hi; i += 32) eq += abs_key(vv[i]) == op.K;
    eq = warp_sum_i(eq);
    warp_offsets(eq, sh);
  }
  const int eq_base = (op.mode == 0) ? sh.woff[threadIdx.x >> 5] : 0;
  const unsigned lt_mask = (1u << lane) - 1u;

  auto wval = [&](float vi, uint32_t key, bool tie_keep) -> float {
    if (op.mode == 0) return (key > op.K || (key == op.K && tie_keep)) ? vi : 0.0f;
    if (key <= op.tkey) return 0.0f;
    if (op.mode == 1) return vi;
    return copysignf(fabsf(vi) - op.tval, vi);
  };
  float part = 0.0f;
  int wnnz = 0;
  {
    int eq_run = eq_base;
    for (int base = sg.lo; base < sg.hi; base += 32) {
      const int i = base + lane;
      const float vi = (i < sg.hi) ? vv[i] : 0.0f;
      const uint32_t key = abs_key(vi);
      bool tie_keep = false;
      if (op.mode == 0) {
        const unsigned b = __ballot_sync(0xffffffffu, i < sg.hi && key == op.K);
        tie_keep = (eq_run + __popc(b & lt_mask)) < op.need_eq;
        eq_run += __popc(b);
      }
      const float w = (i < sg.hi) ? wval(vi, key, tie_keep) : 0.0f;
      part = fmaf(w, w, part);
      wnnz += __popc(__ballot_sync(0xffffffffu, w != 0.0f));
    }
  }
  float fz = 0.0f;
  int zz = 0, nnz_dummy = 0;
  block_sum2f(part, fz, zz, nnz_dummy, sh);
  const double sumsq = (double)part;
  const int nnz = warp_offsets(wnnz, sh);   // sh.woff: each warp's first slot in the support list
  const double nrm = sqrt(sumsq);

  // ---- Table 3 value of the subproblem
  double F;
  if (uses_T(form)) F = nrm;                                   // S3: ||T_s(v)||_2
  else if (uses_lam(form)) F = op.gam * sqrt(a.s) + nrm;       // S4: lambda sqrt(s) + ||V||_2
  else if (uses_U(form)) F = sumsq - op.gam * (double)nnz;     // S5: ||U||^2 - gamma ||U||_0
  else F = nrm;                                                // S6: ||V_gamma(v)||_2

  // ---- pass B
  const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.0f;
  int *gi = sup_idx ? sup_idx + (int64_t)c * a.cap : nullptr;
  float *gv = sup_val ? sup_val + (int64_t)c * a.cap : nullptr;
  {
    int eq_run = eq_base;
    int pos = sh.woff[threadIdx.x >> 5];
    for (int base = sg.lo; base < sg.hi; base += 32) {
      const int i = base + lane;
      const float vi = (i < sg.hi) ? vv[i] : 0.0f;
      const uint32_t key = abs_key(vi);
      bool tie_keep = false;
      if (op.mode == 0) {
        const unsigned b = __ballot_sync(0xffffffffu, i < sg.hi && key == op.K);
        tie_keep = (eq_run + __popc(b & lt_mask)) < op.need_eq;
        eq_run += __popc(b);
      }
      const float w = (i < sg.hi) ? wval(vi, key, tie_keep) : 0.0f;
      const float xi = w * inv;
      const int j = (i < sg.hi) ? (map ? map[i] : i) : 0;
      if (i < sg.hi) x[j] = xi;
      const unsigned nzb = __ballot_sync(0xffffffffu, xi != 0.0f);
      if (gi && xi != 0.0f) {
        const int q = pos + __popc(nzb & lt_mask);
        if (q < a.cap) {
          gi[q] = j;
          gv[q] = xi;
        }
      }
      pos += __popc(nzb);
    }
  }

  // ---- outputs, stopping rule (Section 2.2), control words for the next sweep
  if (threadIdx.x == 0) {
    if (st.F) st.F[c] = F;
    if (st.nnz) st.nnz[c] = nnz;
    if (st.gamma) st.gamma[c] = op.gam;
    if (st.tprev) st.tprev[c] = op.tnext;
    if (st.status) {
      int status = ST_ACTIVE;
      if (nrm == 0.0) {
        status = SPCA_ST_DEGENERATE;
      } else if (a.stop_test && F <= (1.0 + a.tol) * st.F_prev[c]) {
        status = SPCA_ST_CONVERGED;
      } else if (st.iters[c] >= a.max_iter) {
        status = SPCA_ST_MAXITER;
      }
      st.F_prev[c] = F;
      st.status[c] = status;
      // (the active count and list for the next sweep are built after this kernel)
      if (status == ST_ACTIVE && ctrl && nnz > a.sparse_cap) atomicOr(&ctrl->need_dense, 1);
    }
  }
}

// ---------------------------------------------------------------- full x-step
// the full x-step of start c (block-wide; vsm: p floats of shared memory, or null to read v from
// global memory)
__device__ void xstep_full_one(const XstepArgs &a_in, int c, const float *__restrict__ V, int64_t ldv,
                               float *__restrict__ X, int64_t ldx, StartState &st, int *__restrict__ sup_idx,
                               float *__restrict__ sup_val, Ctrl *ctrl, float *vsm, XShared &sh) {
  const bool kSmem = vsm != nullptr;
  const XstepArgs a = xstep_switches(a_in, st.iters, c);
  const int p = a.p;
  const int lane = threadIdx.x & 31;
  const float *vg = V + (int64_t)c * ldv;
  float *x = X + (int64_t)c * ldx;
  const int form = a.form;
  if (kSmem) {
    for (int i = threadIdx.x; i < p; i += XT) vsm[i] = vg[i];
    __syncthreads();
  }
  const float *vv = kSmem ? vsm : vg;
  const Seg sg = warp_seg(p);

  XOp op;
  const int s_int = (int)a.s;
  if (uses_T(form)) {
    op.mode = 1;
    if (s_int < p) {
      bool whole;
      int eq_total;
      radix_select(vv, p, s_int, false, sh, &op.K, &whole, &op.need_eq, &eq_total);
      op.tnext = __uint_as_float(op.K);
      if (whole) {
        op.tkey = op.K == 0u ? 0u : op.K - 1u;   // keep every key >= the bin's lower bound
      } else if (op.K == 0u || op.need_eq >= eq_total) {
        op.tkey = op.K == 0u ? 0u : op.K - 1u;   // no ties to break: keep key >= K
      } else {
        op.mode = 0;
      }
    }
  } else if (uses_lam(form)) {
    // phi(0) = s ||v||_2^2 - ||v||_1^2 >= 0: the L1 ball is not binding, lambda = 0
    float f1 = 0.0f, f2 = 0.0f;
    unsigned mk = 0u;
    for (int i = sg.lo + lane; i < sg.hi; i += 32) {
      const float av = fabsf(vv[i]);
      f1 += av;
      f2 = fmaf(av, av, f2);
      mk = max(mk, __float_as_uint(av));
    }
    int d0 = 0, d1 = 0;
    block_sum2f(f1, f2, d0, d1, sh);
    const uint32_t maxkey = block_max_u(mk, sh.red_u);
    op.mode = 2;
    if ((float)a.s * f2 - f1 * f1 < 0.0f) {
      uint32_t lo;
      op.gam = lambda_s_bisect(vv, p, a.s, 0u, maxkey, sh, &lo);
      op.tkey = lo;
      op.tval = (float)op.gam;
      op.tnext = op.tval;
    }
  } else {  // penalties
    op.mode = uses_U(form) ? 1 : 2;
    if (a.calibrate) {
      const int j = s_int + 1;
      uint32_t tk = 0u;
      if (j <= p) {
        int ne, et;
        bool whole;
        radix_select(vv, p, j, true, sh, &tk, &whole, &ne, &et);
      }
      op.tkey = tk;
      op.tval = __uint_as_float(tk);
      op.gam = uses_U(form) ? (double)op.tval * (double)op.tval : (double)op.tval;
      op.tnext = op.tval;
      if (threadIdx.x == 0 && st.thr) st.thr[c] = op.tval;
    } else if (a.per_start_thr) {
      op.tval = st.thr[c];
      op.gam = st.gamma[c];
      op.tkey = __float_as_uint(op.tval);
    } else {
      op.tval = a.thr_fixed;
      op.gam = a.gamma_fixed;
      op.tkey = __float_as_uint(op.tval);
    }
  }
  xstep_finish(a, c, vv, p, nullptr, op, x, st, sup_idx, sup_val, ctrl, sh);
}

// Every pass over all p entries of v (staged in shared memory when it fits), persistent CTAs over
// the starts.  Starts that the candidate kernels below already finished in this sweep are skipped.
template <bool kSmem>
__global__ void __launch_bounds__(XT) k_xstep(XstepArgs a_in, const float *__restrict__ V, int64_t ldv, int r,
                                              float *__restrict__ X, int64_t ldx, StartState st,
                                              int *__restrict__ sup_idx, float *__restrict__ sup_val,
                                              Ctrl *ctrl) {
  extern __shared__ float vsm[];
  __shared__ XShared sh;
  for (int c = blockIdx.x; c < r; c += gridDim.x) {
    if (st.status && st.status[c] != ST_ACTIVE) continue;
    if (st.xfast && st.xfast[c]) continue;
    xstep_full_one(a_in, c, V, ldv, X, ldx, st, sup_idx, sup_val, ctrl, kSmem ? vsm : nullptr, sh);
    __syncthreads();   // shared memory is reused by the next start
  }
}


// ---------------------------------------------------------------- one-warp operator
// After the candidate filter a start's surviving entries are few (at most kCand) and sit in
// shared memory: one warp finishes the x-step without block barriers.

// the j-th largest key among the |v_i| of vv[0 .. len), 1 <= j <= len, built bit by bit from
// the top (K = the largest key with at least j keys >= K); *n_gt = #(key > K), *n_eq = #(key == K)
__device__ uint32_t warp_select(const float *vv, int len, int j, int *n_gt, int *n_eq) {
  const int lane = threadIdx.x & 31;
  uint32_t K = 0u;
  for (int bit = 30; bit >= 0; --bit) {
    const uint32_t cand = K | (1u << bit);
    int cnt = 0;
    for (int i = lane; i < len; i += 32) cnt += abs_key(vv[i]) >= cand;
    if (warp_sum_i(cnt) >= j) K = cand;
  }
  int gt = 0, eq = 0;
  for (int i = lane; i < len; i += 32) {
    const uint32_t k = abs_key(vv[i]);
    gt += k > K;
    eq += k == K;
  }
  *n_gt = warp_sum_i(gt);
  *n_eq = warp_sum_i(eq);
  return K;
}

// lambda_s over vv[0 .. len) when phi(key lo0) < 0 is known: the bisection and exact root of
// lambda_s_bisect, with warp sums
__device__ double warp_lambda_s(const float *vv, int len, double s, uint32_t lo0, uint32_t maxkey,
                                uint32_t *lo_out) {
  const int lane = threadIdx.x & 31;
  uint32_t lo = lo0, hi = maxkey;
  while (hi - lo > 1u) {
    const uint32_t mid = lo + (hi - lo) / 2u;
    const float lam = __uint_as_float(mid);
    float sw = 0.0f, sw2 = 0.0f;
    int in_lo = 0, in_hi = 0;
    for (int i = lane; i < len; i += 32) {
      const float a = fabsf(vv[i]);
      const uint32_t key = __float_as_uint(a);
      if (a > lam) {
        const float w = a - lam;
        sw += w;
        sw2 = fmaf(w, w, sw2);
      }
      in_lo += (key > lo && key < mid);
      in_hi += (key > mid && key < hi);
    }
    sw = warp_sum_f(sw);
    sw2 = warp_sum_f(sw2);
    in_lo = warp_sum_i(in_lo);
    in_hi = warp_sum_i(in_hi);
    const float phi = (float)s * sw2 - sw * sw;
    if (phi < 0.0f) {
      lo = mid;
      if (in_hi == 0) break;
    } else {
      hi = mid;
      if (in_lo == 0) break;
    }
  }
  float a1 = 0.0f, c1 = 0.0f, a2 = 0.0f, c2 = 0.0f;
  int kc = 0;
  for (int i = lane; i < len; i += 32) {
    const float a = fabsf(vv[i]);
    if (__float_as_uint(a) > lo) {
      ++kc;
      kahan_add(a1, c1, a);
      const float aa = a * a;
      kahan_add(a2, c2, aa);
      kahan_add(a2, c2, fmaf(a, a, -aa));
    }
  }
  const double s1 = warp_sum_d((double)a1 + (double)c1), s2 = warp_sum_d((double)a2 + (double)c2);
  const double k = (double)warp_sum_i(kc);
  const double flo = (double)__uint_as_float(lo), fhi = (double)__uint_as_float(hi);
  double lam;
  if (k <= s) {
    lam = flo;
  } else {
    double disc = s * (k * s2 - s1 * s1) / (k - s);
    if (disc < 0.0) disc = 0.0;
    lam = (s1 - sqrt(disc)) / k;
    lam = fmin(fmax(lam, flo), fhi);
  }
  *lo_out = lo;
  return lam;
}

// xstep_finish for one warp over vv[0 .. len) (element i is entry map[i]): ||w||, nnz, F, x on
// the candidates, the support list in index order, the per-start outputs and the stopping rule
__device__ void xstep_finish_warp(const XstepArgs &a, int c, const float *vv, int len, const int *map, const XOp &op,
                                  float *x, StartState st, int *sup_idx, float *sup_val, Ctrl *ctrl) {
  const int lane = threadIdx.x & 31;
  const int form = a.form;
  const unsigned lt_mask = (1u << lane) - 1u;
  auto wval = [&](float vi, uint32_t key, bool tie_keep) -> float {
    if (op.mode == 0) return (key > op.K || (key == op.K && tie_keep)) ? vi : 0.0f;
    if (key <= op.tkey) return 0.0f;
    if (op.mode == 1) return vi;
    return copysignf(fabsf(vi) - op.tval, vi);
  };
  float part = 0.0f;
  int nnz = 0;
  {
    int eq_run = 0;
    for (int base = 0; base < len; base += 32) {
      const int i = base + lane;
      const float vi = i < len ? vv[i] : 0.0f;
      const uint32_t key = abs_key(vi);
      bool tie_keep = false;
      if (op.mode == 0) {
        const unsigned b = __ballot_sync(0xffffffffu, i < len && key == op.K);
        tie_keep = (eq_run + __popc(b & lt_mask)) < op.need_eq;
        eq_run += __popc(b);
      }
      const float w = i < len ? wval(vi, key, tie_keep) : 0.0f;
      part = fmaf(w, w, part);
      nnz += __popc(__ballot_sync(0xffffffffu, w != 0.0f));
    }
  }
  const double sumsq = (double)warp_sum_f(part);
  const double nrm = sqrt(sumsq);
  double F;
  if (uses_T(form)) F = nrm;
  else if (uses_lam(form)) F = op.gam * sqrt(a.s) + nrm;
  else if (uses_U(form)) F = sumsq - op.gam * (double)nnz;
  else F = nrm;
  const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.0f;
  int *gi = sup_idx + (int64_t)c * a.cap;
  float *gv = sup_val + (int64_t)c * a.cap;
  {
    int eq_run = 0, pos = 0;
    for (int base = 0; base < len; base += 32) {
      const int i = base + lane;
      const float vi = i < len ? vv[i] : 0.0f;
      const uint32_t key = abs_key(vi);
      bool tie_keep = false;
      if (op.mode == 0) {
        const unsigned b = __ballot_sync(0xffffffffu, i < len && key == op.K);
        tie_keep = (eq_run + __popc(b & lt_mask)) < op.need_eq;
        eq_run += __popc(b);
      }
      const float w = i < len ? wval(vi, key, tie_keep) : 0.0f;
      const float xi = w * inv;
      if (i < len) x[map[i]] = xi;
      const unsigned nzb = __ballot_sync(0xffffffffu, xi != 0.0f);
      if (xi != 0.0f) {
        const int q = pos + __popc(nzb & lt_mask);
        if (q < a.cap) {
          gi[q] = map[i];
          gv[q] = xi;
        }
      }
      pos += __popc(nzb);
    }
  }
  if (lane == 0) {
    st.F[c] = F;
    st.nnz[c] = nnz;
    st.gamma[c] = op.gam;
    st.tprev[c] = op.tnext;
    int status = ST_ACTIVE;
    if (nrm == 0.0) {
      status = SPCA_ST_DEGENERATE;
    } else if (a.stop_test && F <= (1.0 + a.tol) * st.F_prev[c]) {
      status = SPCA_ST_CONVERGED;
    } else if (st.iters[c] >= a.max_iter) {
      status = SPCA_ST_MAXITER;
    }
    st.F_prev[c] = F;
    st.status[c] = status;
    if (status == ST_ACTIVE && ctrl && nnz > a.sparse_cap) atomicOr(&ctrl->need_dense, 1);
  }
}

// ---------------------------------------------------------------- candidate x-step
// Near convergence v moves little between sweeps, and every operator keeps only entries above a
// threshold (the s-th or (s+1)-th largest |v_i|, lambda_s, or the penalty's fixed threshold).
// One coalesced pass keeps the entries above a guess in per-warp lists (index order) and sums
// |v| and v^2 for the lambda test; the operator then runs on the candidates in shared memory, and
// x (zero outside the last support list) changes only on the old and the new support.  A guess G
// is valid when the operator's threshold lies above it: at least s (or s + 1) candidates for the
// selections, phi(G) < 0 for lambda_s (phi increases through its root); then the candidates hold
// every surviving entry and the result is the full pass's.
// Two guesses from last sweep's threshold t: the filter keeps the entries above G_lo = kGuessLo t
// while every warp's list has room, and above G_hi = kGuess t otherwise (a warp whose list would
// overflow drops its entries at or below G_hi and goes on with G_hi; then every warp does).  The
// operator takes G_hi when it is valid (fewer candidates) and G_lo otherwise: early sweeps, where
// the threshold can fall by more than a few per cent, then still avoid the full pass.  A start
// whose last sweep took G_hi and moved its threshold by less than kSteady filters with G_hi alone.
// A penalty with its threshold fixed uses that threshold alone (exact).  When no guess is valid,
// or a list overflows at G_hi, the start is left to k_xstep (xfast[c] = 0; otherwise 1 for G_hi
// with a steady threshold, 2 for the rest).
constexpr int kCandW = 64;               // candidates per warp
constexpr int kCand = kCandW * XW;       // per start
static_assert(kCand == kXstepCand, "candidate scratch size");
constexpr float kGuess = 0.85f;
constexpr float kGuessLo = 0.6f;
constexpr float kSteady = 0.05f;         // |t_new / t - 1| below this: one guess next sweep
constexpr int kCandMinP = 4096;          // shorter v: the full pass only
static_assert(kCandMinPGroup <= kCandMinP, "the group's candidate threshold");
constexpr int kMetaHi = 1, kMetaLo = 2;  // meta[c].w: the list holds the entries above G_hi / G_lo

// the candidate x-step's per-start prelude: the guesses (exact: G_hi = G_lo = the threshold
// itself), the number of candidates the operator needs, and whether the filter applies at all
struct CandPlan {
  XstepArgs a;
  float G, Glo, t;
  bool exact, usable;
  int need, s_int;
};
__device__ __forceinline__ CandPlan cand_plan(const XstepArgs &a_in, const StartState &st, int c, bool lists) {
  CandPlan q;
  q.a = xstep_switches(a_in, st.iters, c);
  const int p = q.a.p, form = q.a.form;
  q.s_int = (int)q.a.s;
  q.exact = false;
  if (is_pen(form) && !q.a.calibrate) {
    q.exact = true;
    q.G = q.a.per_start_thr ? st.thr[c] : q.a.thr_fixed;
    q.Glo = q.G;
    q.t = q.G;
  } else {
    // one guess while the threshold holds steady (last sweep took G_hi and moved the threshold
    // by less than kSteady: xfast == 1), two otherwise (the first sweeps, after a G_lo or a full
    // pass, and while the threshold still moves)
    const float t = st.tprev[c];
    q.t = t;
    q.G = kGuess * t;
    q.Glo = st.xfast[c] == 1 ? q.G : kGuessLo * t;
  }
  q.need = uses_T(form) ? q.s_int : (is_pen(form) && q.a.calibrate ? q.s_int + 1 : 1);
  // x is zero outside the last x-step's support list, so only that list is cleared; after the
  // start init (first sweep) x is dense and there is no list: the full pass writes all of x
  q.usable = !((!q.exact && !(q.Glo > 0.0f)) || q.need > p || (uses_T(form) && q.s_int >= p) || st.iters[c] <= 1 ||
               !lists || st.nnz[c] > q.a.cap);
  return q;
}

// keep the entries of a warp's list (val, idx)[0 .. len) whose key is above Gk, in order, in place;
// returns the new length (every lane)
__device__ __forceinline__ int warp_compact_above(float *val, int *idx, int len, uint32_t Gk) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int out = 0;
  __syncwarp();     // the list's entries written by other lanes are visible
  for (int base = 0; base < len; base += 32) {
    const int t = base + lane;
    float v = 0.0f;
    int ix = 0;
    bool keep = false;
    if (t < len) {
      v = val[t];
      ix = idx[t];
      keep = abs_key(v) > Gk;
    }
    const unsigned b = __ballot_sync(0xffffffffu, keep);
    __syncwarp();   // every lane has read its entry before any is overwritten
    if (keep) {     // slot <= t: entries of later rounds are untouched
      const int q = out + __popc(b & lt);
      val[q] = v;
      idx[q] = ix;
    }
    out += __popc(b);
    __syncwarp();
  }
  return out;
}

// Filter: one coalesced pass keeps the entries above the guess in per-warp lists, concatenated in
// warp order (the candidates in index order) into cand_val / cand_idx (kCand per start), with the
// sums of |v| and v^2 (lambda forms) and the count in meta[c]; x is cleared on the last support.
// A start the filter cannot serve gets xfast[c] = 0 and meta[c].w = 0.
constexpr int kFilterChunks = 4;      // 128-entry chunks per warp and step, loaded before use
constexpr int kFilterMinBlocks = 2;   // resident CTAs per SM the register budget is set for
// shared memory of the filter (one CTA per start)
struct FilterShared {
  XShared sh;
  float wval_s[kCand];
  int widx_s[kCand];
  int fail_s, raised_s;
};
// start c: its candidates go to gv / gi (kCand each) and its counts to *meta_c
__device__ __forceinline__ void xstep_filter_one(const XstepArgs &a_in, int c, const float *__restrict__ V,
                                                 int64_t ldv, float *__restrict__ X, int64_t ldx,
                                                 const StartState &st, const int *__restrict__ sup_idx,
                                                 float *__restrict__ gv, int *__restrict__ gi, int4 *meta_c,
                                                 FilterShared &fs) {
  XShared &sh = fs.sh;
  float *wval_s = fs.wval_s;
  int *widx_s = fs.widx_s;
  int &fail_s = fs.fail_s, &raised_s = fs.raised_s;
  if (st.status[c] != ST_ACTIVE) return;
  const CandPlan q = cand_plan(a_in, st, c, sup_idx != nullptr);
  if (!q.usable) {
    if (threadIdx.x == 0) {
      st.xfast[c] = 0;
      meta_c->w = 0;
    }
    return;
  }
  const int p = q.a.p;
  const bool sums = uses_lam(q.a.form);   // |v| and v^2 sums: the lambda forms' phi(0) test
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t Ghi = __float_as_uint(q.G);
  uint32_t Gk = __float_as_uint(q.Glo);   // the warp's current guess (warp-uniform)
  bool raised = Gk == Ghi;
  // kFilterChunks 128-entry chunks per step, their loads issued before any is used
  const float *vg = V + (int64_t)c * ldv;
  float *x = X + (int64_t)c * ldx;
  const int seg = ((p + XW - 1) / XW + 127) / 128 * 128;
  const int lo = min(p, w * seg), hi = min(p, lo + seg);
  float *wv = wval_s + w * kCandW;
  int *wi = widx_s + w * kCandW;
  int wc = 0;
  bool over = false;
  float f1 = 0.0f, f2 = 0.0f;
  for (int base = lo; base < hi && !over; base += 128 * kFilterChunks) {
    float e[kFilterChunks][4];
    const bool full = base + 128 * kFilterChunks <= hi;
#pragma unroll
    for (int h = 0; h < kFilterChunks; ++h) {
      const int i0 = base + h * 128 + 4 * lane;
      if (full || i0 + 3 < hi) {
        const float4 t = *reinterpret_cast<const float4 *>(vg + i0);
        e[h][0] = t.x; e[h][1] = t.y; e[h][2] = t.z; e[h][3] = t.w;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) e[h][k] = (i0 + k < hi) ? vg[i0 + k] : 0.0f;   // 0 is never kept
      }
    }
#pragma unroll
    for (int h = 0; h < kFilterChunks; ++h) {
      const int i0 = base + h * 128 + 4 * lane;
      if (sums) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float av = fabsf(e[h][k]);
          f1 += av;
          f2 = fmaf(av, av, f2);
        }
      }
      int cnt = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) cnt += abs_key(e[h][k]) > Gk ? 1 : 0;
      if (!__any_sync(0xffffffffu, cnt != 0)) continue;   // the common case: nothing above the guess
      // the warp's exclusive prefix of cnt (0..4) from the ballots of its three bits
      unsigned b0 = __ballot_sync(0xffffffffu, cnt & 1), b1 = __ballot_sync(0xffffffffu, cnt & 2),
               b2 = __ballot_sync(0xffffffffu, cnt & 4);
      int tot = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
      if (wc + tot > kCandW && !raised) {   // no room at G_lo: keep only the entries above G_hi
        wc = warp_compact_above(wv, wi, wc, Ghi);
        Gk = Ghi;
        raised = true;
        cnt = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) cnt += abs_key(e[h][k]) > Gk ? 1 : 0;
        b0 = __ballot_sync(0xffffffffu, cnt & 1);
        b1 = __ballot_sync(0xffffffffu, cnt & 2);
        b2 = __ballot_sync(0xffffffffu, cnt & 4);
        tot = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
      }
      if (wc + tot > kCandW) {
        over = true;
        break;
      }
      int q2 = wc + __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (abs_key(e[h][k]) > Gk) {
          wv[q2] = e[h][k];
          wi[q2] = i0 + k;
          ++q2;
        }
      }
      wc += tot;
    }
  }
  if (threadIdx.x == 0) {
    fail_s = 0;
    raised_s = 0;
  }
  __syncthreads();
  if (lane == 0 && over) fail_s = 1;
  if (lane == 0 && Gk != __float_as_uint(q.Glo)) raised_s = 1;   // this warp went on with G_hi
  int d0 = 0, d1 = 0;
  block_sum2f(f1, f2, d0, d1, sh);   // (its barriers also publish fail_s and raised_s)
  if (fail_s) {
    if (threadIdx.x == 0) {
      st.xfast[c] = 0;
      meta_c->w = 0;
    }
    return;
  }
  const bool at_hi = raised_s || Ghi == __float_as_uint(q.Glo);
  __syncwarp();
  if (at_hi && Gk != Ghi) wc = warp_compact_above(wv, wi, wc, Ghi);   // every warp on one guess
  const int ncand = warp_offsets(lane == 0 ? wc : 0, sh);
  const int off = sh.woff[w];
  for (int t = lane; t < wc; t += 32) {
    gv[off + t] = wv[t];
    gi[off + t] = wi[t];
  }
  const int nnz_old = st.nnz[c];
  const int *old = sup_idx + (int64_t)c * q.a.cap;
  for (int t = threadIdx.x; t < nnz_old; t += XT) x[old[t]] = 0.0f;
  if (threadIdx.x == 0)
    *meta_c = make_int4(ncand, __float_as_int(f1), __float_as_int(f2), at_hi ? kMetaHi : kMetaLo);
}

__global__ void __launch_bounds__(XT, kFilterMinBlocks) k_xstep_filter(XstepArgs a_in, const float *__restrict__ V, int64_t ldv,
                                                     float *__restrict__ X, int64_t ldx, StartState st,
                                                     const int *__restrict__ sup_idx, float *__restrict__ cand_val,
                                                     int *__restrict__ cand_idx, int4 *__restrict__ meta) {
  __shared__ FilterShared fs;
  const int c = blockIdx.x;
  xstep_filter_one(a_in, c, V, ldv, X, ldx, st, sup_idx, cand_val + (int64_t)c * kCand, cand_idx + (int64_t)c * kCand,
                   meta + c, fs);
}

// Operator: a warp per start on the filter's candidates (staged in the warp's shared memory).
// A list above G_lo is first cut to the entries above G_hi when G_hi is valid; then the operator,
// with the check that the guess lies below the operator's threshold, the new x, F and support.
constexpr int kOpWarps = 4;
// start c on one warp: its candidates at gv / gi, its counts at *meta_c; cval / cidx: the warp's
// shared memory (kCand each)
__device__ __forceinline__ void xstep_op_one(const XstepArgs &a_in, int c, float *__restrict__ X, int64_t ldx,
                                             const StartState &st, int *__restrict__ sup_idx,
                                             float *__restrict__ sup_val, const float *__restrict__ gv,
                                             const int *__restrict__ gi, const int4 *meta_c, Ctrl *ctrl, float *cval,
                                             int *cidx) {
  const int lane = threadIdx.x & 31;
  if (st.status[c] != ST_ACTIVE) return;
  const int4 m = *meta_c;
  if (m.w == 0) return;
  const CandPlan q = cand_plan(a_in, st, c, true);
  const XstepArgs &a = q.a;
  const int form = a.form, s_int = q.s_int;
  int ncand = m.x;
  const float f1 = __int_as_float(m.y), f2 = __int_as_float(m.z);
  for (int t = lane; t < ncand; t += 32) {
    cval[t] = gv[t];
    cidx[t] = gi[t];
  }
  __syncwarp();
  // phi(G) < 0 over the candidates above G (all of v's entries above G when the list holds them)
  auto phi_below = [&](float G, int len) {
    const uint32_t Gk = __float_as_uint(G);
    float sw = 0.0f, sw2 = 0.0f;
    for (int i = lane; i < len; i += 32) {
      const float av = fabsf(cval[i]);
      if (__float_as_uint(av) > Gk) {
        const float wv2 = av - G;
        sw += wv2;
        sw2 = fmaf(wv2, wv2, sw2);
      }
    }
    sw = warp_sum_f(sw);
    sw2 = warp_sum_f(sw2);
    return (float)a.s * sw2 - sw * sw < 0.0f;
  };
  float G = q.G;
  if (m.w == kMetaLo) {   // the list holds the entries above G_lo: cut it to G_hi if G_hi is valid
    const uint32_t Ghi = __float_as_uint(q.G);
    bool hi_ok;
    if (uses_lam(form)) {
      hi_ok = phi_below(q.G, ncand);
    } else {
      int n_hi = 0;
      for (int i = lane; i < ncand; i += 32) n_hi += abs_key(cval[i]) > Ghi ? 1 : 0;
      hi_ok = warp_sum_i(n_hi) >= q.need;
    }
    if (hi_ok) ncand = warp_compact_above(cval, cidx, ncand, Ghi);
    else G = q.Glo;
  }
  const uint32_t Gk = __float_as_uint(G);
  float *x = X + (int64_t)c * ldx;
  XOp op;
  bool ok = ncand >= q.need;
  if (ok && uses_T(form)) {
    int gt, eq;
    op.K = warp_select(cval, ncand, s_int, &gt, &eq);
    op.need_eq = s_int - gt;
    op.tnext = __uint_as_float(op.K);
    if (op.need_eq >= eq) {   // every key equal to K is kept: keep key >= K
      op.mode = 1;
      op.tkey = op.K - 1u;
    } else {
      op.mode = 0;            // ties at K: the first need_eq in index order
    }
  } else if (ok && uses_lam(form)) {
    // lambda = 0 (phi(0) >= 0) keeps every entry: left to the full pass
    ok = (float)a.s * f2 - f1 * f1 < 0.0f;
    if (ok) ok = phi_below(G, ncand);   // phi(G) < 0: lambda_s > G
    if (ok) {
      unsigned mk = 0u;
      for (int i = lane; i < ncand; i += 32) mk = max(mk, abs_key(cval[i]));
      mk = warp_max_u(mk);
      uint32_t lok;
      op.mode = 2;
      op.gam = warp_lambda_s(cval, ncand, a.s, Gk, mk, &lok);
      op.tkey = lok;
      op.tval = (float)op.gam;
      op.tnext = op.tval;
    }
  } else if (ok) {  // penalties
    op.mode = uses_U(form) ? 1 : 2;
    if (a.calibrate) {
      int gt, eq;
      const uint32_t tk = warp_select(cval, ncand, s_int + 1, &gt, &eq);   // the (s+1)-th largest
      op.tkey = tk;
      op.tval = __uint_as_float(tk);
      op.gam = uses_U(form) ? (double)op.tval * (double)op.tval : (double)op.tval;
      op.tnext = op.tval;
      if (lane == 0) st.thr[c] = op.tval;
    } else if (a.per_start_thr) {
      op.tval = st.thr[c];
      op.gam = st.gamma[c];
      op.tkey = __float_as_uint(op.tval);
      op.tnext = st.tprev[c];
    } else {
      op.tval = a.thr_fixed;
      op.gam = a.gamma_fixed;
      op.tkey = __float_as_uint(op.tval);
      op.tnext = st.tprev[c];
    }
  }
  if (!ok) {   // uniform over the warp: every input of ok is a warp-wide value
    if (lane == 0) st.xfast[c] = 0;
    return;
  }
  xstep_finish_warp(a, c, cval, ncand, cidx, op, x, st, sup_idx, sup_val, ctrl);
  if (lane == 0) {   // 1: G_hi taken and the threshold steady (a fixed threshold counts as steady)
    const bool steady = q.exact || (op.tnext >= (1.0f - kSteady) * q.t && op.tnext <= (1.0f + kSteady) * q.t);
    st.xfast[c] = G == q.G && steady ? 1 : 2;
  }
}

__global__ void __launch_bounds__(32 * kOpWarps) k_xstep_op(XstepArgs a_in, int r, float *__restrict__ X,
                                                            int64_t ldx, StartState st, int *__restrict__ sup_idx,
                                                            float *__restrict__ sup_val,
                                                            const float *__restrict__ cand_val,
                                                            const int *__restrict__ cand_idx,
                                                            const int4 *__restrict__ meta, Ctrl *ctrl) {
  __shared__ float cval_s[kOpWarps][kCand];
  __shared__ int cidx_s[kOpWarps][kCand];
  const int w = threadIdx.x >> 5;
  const int c = blockIdx.x * kOpWarps + w;
  if (c >= r) return;
  xstep_op_one(a_in, c, X, ldx, st, sup_idx, sup_val, cand_val + (int64_t)c * kCand, cand_idx + (int64_t)c * kCand,
               meta + c, ctrl, cval_s[w], cidx_s[w]);
}
}  // namespace

// groups of problems: the full pass for every active start of every problem, persistent CTAs over
// the global starts; the kSmem launch takes the problems whose v fits in shared memory (staged
// there), the other launch the rest
template <bool kSmem>
__global__ void __launch_bounds__(XT, 2) k_g_xstep(const GProb *__restrict__ P, const int *__restrict__ prob, int R,
                                                   int parity, int cand) {
  extern __shared__ float vsm[];
  __shared__ XShared sh;
  for (int g = blockIdx.x; g < R; g += gridDim.x) {
    const GProb &q = P[prob[g]];
    if (kSmem != ((size_t)q.p * sizeof(float) <= (size_t)XSTEP_SMEM_MAX)) continue;
    const int c = g - q.start0;
    StartState st = q.st;
    if (st.status[c] != ST_ACTIVE) continue;
    if (cand && st.xfast[c]) continue;   // the candidate kernels finished it this sweep
    st.xfast = nullptr;
    xstep_full_one(q.xa, c, q.V, q.ldX, q.X, q.ldX, st, q.sup_idx, q.sup_val, q.ctrl[parity], kSmem ? vsm : nullptr,
                   sh);
    __syncthreads();   // shared memory is reused by the next start
  }
}

// groups of problems: the candidate kernels for every active start of every problem, as in
// launch_xstep (a CTA per global start for the filter, a warp per global start for the operator);
// a problem whose v is shorter than kCandMinPGroup is left to the full pass (xfast = 0).  The
// threshold is lower than a single problem's kCandMinP: a group's launches are shared by all its
// starts, so the filter and operator cost no launches of their own per problem.
__global__ void __launch_bounds__(XT, kFilterMinBlocks) k_g_xstep_filter(const GProb *__restrict__ P,
                                                                         const int *__restrict__ prob) {
  __shared__ FilterShared fs;
  const GProb &q = P[prob[blockIdx.x]];
  const int c = (int)blockIdx.x - q.start0;
  if (q.p < kCandMinPGroup) {
    if (threadIdx.x == 0 && q.st.status[c] == ST_ACTIVE) {
      q.st.xfast[c] = 0;
      q.meta[c].w = 0;
    }
    return;
  }
  xstep_filter_one(q.xa, c, q.V, q.ldX, q.X, q.ldX, q.st, q.sup_idx, q.cand_val + (int64_t)c * kCand,
                   q.cand_idx + (int64_t)c * kCand, q.meta + c, fs);
}

__global__ void __launch_bounds__(32 * kOpWarps) k_g_xstep_op(const GProb *__restrict__ P, const int *__restrict__ prob,
                                                              int R, int parity) {
  __shared__ float cval_s[kOpWarps][kCand];
  __shared__ int cidx_s[kOpWarps][kCand];
  const int w = threadIdx.x >> 5;
  const int g = blockIdx.x * kOpWarps + w;
  if (g >= R) return;
  const GProb &q = P[prob[g]];
  if (q.p < kCandMinPGroup) return;
  const int c = g - q.start0;
  xstep_op_one(q.xa, c, q.X, q.ldX, q.st, q.sup_idx, q.sup_val, q.cand_val + (int64_t)c * kCand,
               q.cand_idx + (int64_t)c * kCand, q.meta + c, q.ctrl[parity], cval_s[w], cidx_s[w]);
}

cudaError_t launch_g_xstep(const GProb *P, const int *prob, int R, int max_p_small, bool any_large, bool cand,
                           int parity, int sms, cudaStream_t st) {
  if (cand) {
    k_g_xstep_filter<<<R, XT, 0, st>>>(P, prob);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_g_xstep_op<<<(R + kOpWarps - 1) / kOpWarps, 32 * kOpWarps, 0, st>>>(P, prob, R, parity);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (max_p_small > 0) {   // the problems whose v fits in shared memory: staged there
    const size_t bytes = (size_t)max_p_small * sizeof(float);
    if (bytes > (size_t)XSTEP_SMEM_MAX) return cudaErrorInvalidValue;
    static const cudaError_t configured =
        cudaFuncSetAttribute(k_g_xstep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, XSTEP_SMEM_MAX);
    if (configured != cudaSuccess) return configured;
    const int per_sm = bytes <= 100u * 1024u ? 2 : 1;
    k_g_xstep<true><<<min(R, per_sm * sms), XT, bytes, st>>>(P, prob, R, parity, cand ? 1 : 0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (any_large) {
    k_g_xstep<false><<<min(R, 2 * sms), XT, 0, st>>>(P, prob, R, parity, cand ? 1 : 0);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------- small problems in one launch
// For a small matrix the chain of launches of a sweep, not its work, sets the time.  Here every
// sweep of a start runs in one CTA, all starts at once (a CTA per start): u = A x as a warp per
// row of A, v = A^T y as a thread per column of A (both on the CUDA cores, sums in a fixed order;
// A stays in L2 across the sweeps), then the y-step and the full-pass x-step of the
// single-problem path, until the start stops or `sweeps` sweeps have run.  x and y are staged in
// shared memory; v too, for the x-step.
__global__ void __launch_bounds__(XT) k_small_sweeps(XstepArgs xa, const float *__restrict__ A, int64_t lda, int n,
                                                     int p, float *__restrict__ X, int64_t ldx, float *__restrict__ U,
                                                     float *__restrict__ Y, int64_t ldu, float *__restrict__ V,
                                                     StartState st, int *__restrict__ sup_idx,
                                                     float *__restrict__ sup_val, int sweeps) {
  extern __shared__ float4 sm4[];
  float *sm = reinterpret_cast<float *>(sm4);
  __shared__ XShared sh;
  __shared__ float redf[32];
  const int c = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p4 = (p + 3) & ~3, n4 = (n + 3) & ~3;
  float *xs = sm;              // x (p), then y (n) in the same place
  float *vsm = sm + max(p4, n4);
  const float *x = X + (int64_t)c * ldx;
  float *u = U + (int64_t)c * ldu;
  const float *y = Y + (int64_t)c * ldu;
  float *v = V + (int64_t)c * ldx;
  for (int k = 0; k < sweeps; ++k) {
    __syncthreads();   // (the status and x written by the last x-step)
    if (st.status[c] != ST_ACTIVE) break;
    for (int j = threadIdx.x; j < p; j += XT) xs[j] = x[j];
    __syncthreads();
    for (int i = warp; i < n; i += XW) {   // u = A x
      const float *a = A + (int64_t)i * lda;
      float acc = 0.0f;
      for (int j = lane; j < p; j += 32) acc = fmaf(a[j], xs[j], acc);
      acc = warp_sum_f(acc);
      if (lane == 0) u[i] = acc;
    }
    __syncthreads();
    ystep_body(xa.form, U, ldu, n, Y, nullptr, 0, nullptr, st, X, ldx, p, c, redf);
    __syncthreads();
    if (st.status[c] != ST_ACTIVE) break;   // u = 0 under L2 variance: degenerate
    for (int i = threadIdx.x; i < n; i += XT) xs[i] = y[i];
    __syncthreads();
    for (int j = threadIdx.x; j < p; j += XT) {   // v = A^T y, a column of A per thread
      float acc = 0.0f;
      for (int i = 0; i < n; ++i) acc = fmaf(A[(int64_t)i * lda + j], xs[i], acc);
      v[j] = acc;
    }
    __syncthreads();
    xstep_full_one(xa, c, V, ldx, X, ldx, st, sup_idx, sup_val, nullptr, vsm, sh);
  }
}

// (measured on GB300: with one CTA per start, a start's sweep costs about as much as the launch
// chain it replaces at n p ~ 4e5, so mid-sized matrices take this path only with enough starts
// to fill the device)
bool small_sweeps_fit(int64_t n, int64_t p, int r) {
  const int64_t words = ((std::max(n, p) + 3) & ~int64_t(3)) + ((p + 3) & ~int64_t(3));
  if (words * 4 > (int64_t)XSTEP_SMEM_MAX) return false;
  return n * p <= kSmallAlwaysEntries || (n * p <= kSmallMaxEntries && r >= kSmallMinStarts);
}

cudaError_t launch_small_sweeps(XstepArgs xa, const float *A, int64_t lda, int n, int p, float *X, int64_t ldx,
                                float *U, float *Y, int64_t ldu, float *V, StartState s, int *sup_idx, float *sup_val,
                                int r, int sweeps, cudaStream_t st) {
  if (!small_sweeps_fit(n, p, r)) return cudaErrorInvalidValue;
  static const cudaError_t configured =
      cudaFuncSetAttribute(k_small_sweeps, cudaFuncAttributeMaxDynamicSharedMemorySize, XSTEP_SMEM_MAX);
  if (configured != cudaSuccess) return configured;
  const size_t bytes = 4 * (size_t)((((std::max(n, p) + 3) & ~3)) + ((p + 3) & ~3));
  k_small_sweeps<<<r, XT, bytes, st>>>(xa, A, lda, n, p, X, ldx, U, Y, ldu, V, s, sup_idx, sup_val, sweeps);
  return cudaGetLastError();
}

cudaError_t launch_xstep(XstepArgs a, const float *V, int64_t ldv, int r, float *X, int64_t ldx,
                         StartState s, int *sup_idx, float *sup_val, Ctrl *ctrl_next, XstepScratch scratch,
                         cudaStream_t st) {
  // the candidate kernels need the per-start thresholds of the last sweep, 16-byte rows and their
  // scratch (candidate lists, per-start counts)
  // (for short v, p < kCandMinP, the full pass alone is cheaper than three launches)
  const bool cand = a.p >= kCandMinP && s.status && s.tprev && s.xfast && s.thr && ldv % 4 == 0 && ldx % 4 == 0 &&
                    (reinterpret_cast<uintptr_t>(V) & 15u) == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0 &&
                    scratch.cand_val && scratch.cand_idx && scratch.meta;
  if (cand) {
    k_xstep_filter<<<r, XT, 0, st>>>(a, V, ldv, X, ldx, s, sup_idx, scratch.cand_val, scratch.cand_idx,
                                     reinterpret_cast<int4 *>(scratch.meta));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_xstep_op<<<(r + kOpWarps - 1) / kOpWarps, 32 * kOpWarps, 0, st>>>(
        a, r, X, ldx, s, sup_idx, sup_val, scratch.cand_val, scratch.cand_idx,
        reinterpret_cast<const int4 *>(scratch.meta), ctrl_next);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else {
    s.xfast = nullptr;
  }
  // the full pass for the starts the candidate kernels left: persistent CTAs (as many as fit),
  // so that a sweep in which every start took the candidate path costs one short launch
  // (function-local statics: initialised once, thread-safe)
  static const int sms = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
      return 0;
    return v;
  }();
  if (sms < 1) return cudaErrorInvalidDevice;
  const size_t bytes = (size_t)a.p * sizeof(float);
  if (bytes <= (size_t)XSTEP_SMEM_MAX) {
    static const cudaError_t configured =
        cudaFuncSetAttribute(k_xstep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, XSTEP_SMEM_MAX);
    if (configured != cudaSuccess) return configured;
    const int per_sm = bytes <= 100u * 1024u ? 2 : 1;
    k_xstep<true><<<min(r, per_sm * sms), XT, bytes, st>>>(a, V, ldv, r, X, ldx, s, sup_idx, sup_val, ctrl_next);
  } else {
    k_xstep<false><<<min(r, 2 * sms), XT, 0, st>>>(a, V, ldv, r, X, ldx, s, sup_idx, sup_val, ctrl_next);
  }
  return cudaGetLastError();
}

}  // namespace spca
