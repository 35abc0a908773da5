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
#include <cstdint>

#include "block_util.cuh"
#include "spca_internal.cuh"

namespace spca {

namespace {
constexpr int XT = 512;  // threads per CTA

struct XShared {
  unsigned hist[256];
  double red_d[32];
  int red_i[32];
  unsigned red_u[32];
  int digit, rem;
};

// The j-th largest (1 <= j <= p) of the keys |v_i| (MSB-first radix select, 8-bit digits).
// Returns the key; *need_eq = how many elements equal to it belong to the top j, and
// *eq_total = how many elements equal it.
__device__ uint32_t radix_select_desc(const float *__restrict__ v, int p, int j, XShared &sh,
                                      int *need_eq, int *eq_total) {
  uint32_t prefix = 0, mask = 0;
  int rem = j;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int b = threadIdx.x; b < 256; b += blockDim.x) sh.hist[b] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
      const uint32_t key = abs_key(v[i]);
      if ((key & mask) == prefix) atomicAdd(&sh.hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0, d = 255;
      for (; d > 0; --d) {
        if (acc + (int)sh.hist[d] >= rem) break;
        acc += (int)sh.hist[d];
      }
      sh.digit = d;
      sh.rem = rem - acc;
    }
    __syncthreads();
    prefix |= (uint32_t)sh.digit << shift;
    mask |= 255u << shift;
    rem = sh.rem;
    if (shift == 0) *eq_total = (int)sh.hist[sh.digit];
    __syncthreads();
  }
  *need_eq = rem;
  return prefix;
}

// lambda_s(v) (Section 2.1) for the case phi(0) < 0.  Returns lambda and the key interval
// (lo, hi] such that the active set {|v_i| > lambda} = {key_i > lo}.
__device__ double lambda_s_bisect(const float *__restrict__ v, int p, double s, uint32_t maxkey,
                                  XShared &sh, uint32_t *lo_out) {
  uint32_t lo = 0u, hi = maxkey;  // phi(key lo) < 0 <= phi(key hi)
  while (hi - lo > 1u) {
    const uint32_t mid = lo + (hi - lo) / 2u;
    const float lam = __uint_as_float(mid);
    float sw = 0.0f, sw2 = 0.0f;
    int in_lo = 0, in_hi = 0;  // elements strictly inside (lo, mid) and (mid, hi)
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
      const float a = fabsf(v[i]);
      const uint32_t key = __float_as_uint(a);
      if (a > lam) {
        const float w = a - lam;
        sw += w;
        sw2 = fmaf(w, w, sw2);
      }
      in_lo += (key > lo && key < mid);
      in_hi += (key > mid && key < hi);
    }
    const double Sw = block_sum_d((double)sw, sh.red_d);
    const double Sw2 = block_sum_d((double)sw2, sh.red_d);
    const int nlo = block_sum_i(in_lo, sh.red_i);
    const int nhi = block_sum_i(in_hi, sh.red_i);
    const double phi = s * Sw2 - Sw * Sw;
    if (phi < 0.0) {
      lo = mid;
      if (nhi == 0) break;  // no magnitude strictly inside (mid, hi): active set fixed
    } else {
      hi = mid;
      if (nlo == 0) break;
    }
  }
  // active set {key > lo}: k, S1, S2 in FP64, then the root of phi on this piece
  int kc = 0;
  double s1 = 0.0, s2 = 0.0;
  {
    double d1 = 0.0, d2 = 0.0;
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
      const float a = fabsf(v[i]);
      if (__float_as_uint(a) > lo) {
        ++kc;
        d1 += (double)a;
        d2 = fma((double)a, (double)a, d2);
      }
    }
    s1 = block_sum_d(d1, sh.red_d);
    s2 = block_sum_d(d2, sh.red_d);
    kc = block_sum_i(kc, sh.red_i);
  }
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
}  // namespace

__global__ void __launch_bounds__(XT) k_xstep(XstepArgs a, const float *__restrict__ V, int64_t ldv,
                                              float *__restrict__ X, int64_t ldx, StartState st,
                                              int *__restrict__ sup_idx,
                                              float *__restrict__ sup_val, Ctrl *ctrl) {
  __shared__ XShared sh;
  const int c = blockIdx.x;
  if (st.status && st.status[c] != ST_ACTIVE) return;
  const int p = a.p;
  const float *v = V + (int64_t)c * ldv;
  float *x = X + (int64_t)c * ldx;
  const int form = a.form;

  // ---- choose the operator's parameters
  // mode 0: T_s (keep key > K, plus the first need_eq of key == K in index order)
  // mode 1: hard threshold: keep key > tkey, value v            (U_gamma; T_s with s >= p)
  // mode 2: soft threshold: keep key > tkey, value sgn(v)(|v|-t)  (V_gamma, V_lambda)
  int mode = 0;
  uint32_t K = 0u, tkey = 0u;
  int need_eq = 0, eq_total = 0;
  float tval = 0.0f;     // threshold value subtracted in mode 2
  double gam = 0.0;      // gamma in Table 1 units (penalties) or lambda_s (S4)
  const int s_int = (int)a.s;

  if (uses_T(form)) {
    if (s_int >= p) {
      mode = 1;
      tkey = 0u;
    } else {
      K = radix_select_desc(v, p, s_int, sh, &need_eq, &eq_total);
      if (K == 0u || need_eq >= eq_total) {
        mode = 1;  // no ties to break: keep key >= K (zeros contribute nothing)
        tkey = K == 0u ? 0u : K - 1u;
      }
    }
  } else if (uses_lam(form)) {
    // phi(0) = s ||v||_2^2 - ||v||_1^2 >= 0: the L1 ball is not binding, lambda = 0
    float f1 = 0.0f, f2 = 0.0f;
    unsigned mk = 0u;
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
      const float av = fabsf(v[i]);
      f1 += av;
      f2 = fmaf(av, av, f2);
      mk = max(mk, __float_as_uint(av));
    }
    const double S1 = block_sum_d((double)f1, sh.red_d);
    const double S2 = block_sum_d((double)f2, sh.red_d);
    const uint32_t maxkey = block_max_u(mk, sh.red_u);
    mode = 2;
    if (a.s * S2 - S1 * S1 >= 0.0) {
      gam = 0.0;
      tkey = 0u;
      tval = 0.0f;
    } else {
      uint32_t lo;
      gam = lambda_s_bisect(v, p, a.s, maxkey, sh, &lo);
      tkey = lo;
      tval = (float)gam;
    }
  } else {  // penalties
    mode = uses_U(form) ? 1 : 2;
    if (a.calibrate) {
      const int j = s_int + 1;
      uint32_t tk = 0u;
      if (j <= p) {
        int ne, et;
        tk = radix_select_desc(v, p, j, sh, &ne, &et);
      }
      tkey = tk;
      tval = __uint_as_float(tk);
      gam = uses_U(form) ? (double)tval * (double)tval : (double)tval;
      if (threadIdx.x == 0 && st.thr) st.thr[c] = tval;
    } else if (a.per_start_thr) {
      tval = st.thr[c];
      gam = st.gamma[c];
      tkey = __float_as_uint(tval);
    } else {
      tval = a.thr_fixed;
      gam = a.gamma_fixed;
      tkey = __float_as_uint(tval);
    }
  }

  // ---- pass A: ||w||_2^2 and nnz of the unnormalised result w, in index order
  auto wval = [&](int i, float vi, bool tie_keep) -> float {
    const uint32_t key = abs_key(vi);
    if (mode == 0) return (key > K || (key == K && tie_keep)) ? vi : 0.0f;
    if (key <= tkey) return 0.0f;
    if (mode == 1) return vi;
    return copysignf(fabsf(vi) - tval, vi);
  };
  float part = 0.0f;
  int cnt = 0;
  int eq_seen = 0;
  for (int base = 0; base < p; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const float vi = (i < p) ? v[i] : 0.0f;
    bool tie_keep = false;
    if (mode == 0) {  // rank among equal keys, in index order (block-wide scan)
      int tot;
      const bool eq = (i < p) && abs_key(vi) == K;
      const int rank = eq_seen + block_excl_scan_flag(eq, sh.red_i, &tot);
      tie_keep = eq && rank < need_eq;
      eq_seen += tot;
    }
    const float w = (i < p) ? wval(i, vi, tie_keep) : 0.0f;
    part = fmaf(w, w, part);
    cnt += (w != 0.0f);
  }
  const double sumsq = block_sum_d((double)part, sh.red_d);
  const int nnz = block_sum_i(cnt, sh.red_i);
  const double nrm = sqrt(sumsq);

  // ---- Table 3 value of the subproblem
  double F;
  if (uses_T(form)) F = nrm;                                   // S3: ||T_s(v)||_2
  else if (uses_lam(form)) F = gam * sqrt(a.s) + nrm;          // S4: lambda sqrt(s) + ||V||_2
  else if (uses_U(form)) F = sumsq - gam * (double)nnz;        // S5: ||U||^2 - gamma ||U||_0
  else F = nrm;                                                // S6: ||V_gamma(v)||_2

  // ---- pass B: x = w / ||w||_2, support list in index order
  const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.0f;
  int *gi = sup_idx ? sup_idx + (int64_t)c * a.cap : nullptr;
  float *gv = sup_val ? sup_val + (int64_t)c * a.cap : nullptr;
  int written = 0;
  eq_seen = 0;
  for (int base = 0; base < p; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const float vi = (i < p) ? v[i] : 0.0f;
    bool tie_keep = false;
    if (mode == 0) {
      int tot;
      const bool eq = (i < p) && abs_key(vi) == K;
      const int rank = eq_seen + block_excl_scan_flag(eq, sh.red_i, &tot);
      tie_keep = eq && rank < need_eq;
      eq_seen += tot;
    }
    const float w = (i < p) ? wval(i, vi, tie_keep) : 0.0f;
    const float xi = w * inv;
    if (i < p) x[i] = xi;
    if (gi) {
      int tot;
      const int pos = written + block_excl_scan_flag(xi != 0.0f, sh.red_i, &tot);
      if (xi != 0.0f && pos < a.cap) {
        gi[pos] = i;
        gv[pos] = xi;
      }
      written += tot;
    }
  }

  // ---- outputs, stopping rule (Section 2.2), control words for the next sweep
  if (threadIdx.x == 0) {
    if (st.F) st.F[c] = F;
    if (st.nnz) st.nnz[c] = nnz;
    if (st.gamma) st.gamma[c] = gam;
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
      if (status == ST_ACTIVE && ctrl) {
        atomicAdd(&ctrl->active, 1);
        if (nnz > a.sparse_cap) atomicOr(&ctrl->need_dense, 1);
      }
    }
  }
}

cudaError_t launch_xstep(XstepArgs a, const float *V, int64_t ldv, int r, float *X, int64_t ldx,
                         StartState s, int *sup_idx, float *sup_val, Ctrl *ctrl_next,
                         cudaStream_t st) {
  k_xstep<<<r, XT, 0, st>>>(a, V, ldv, X, ldx, s, sup_idx, sup_val, ctrl_next);
  return cudaGetLastError();
}

}  // namespace spca
