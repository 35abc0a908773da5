/*
 * spca_oracle.c -- plain FP64 CPU oracle for the alternating-maximization (AM) method
 * for the eight single-component sparse PCA formulations of
 *   P. Richtarik, M. Jahani, S. D. Ahipasaoglu, M. Takac,
 *   "Alternating maximization: unifying framework for 8 sparse PCA formulations and
 *    efficient parallel codes" (arXiv 1212.4137).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code with the CUDA path.
 *
 * Everything is FP64, every loop runs in plain index order, and every step follows the
 * paper in its order and notation:
 *   Table 1          the eight problems  OPT = max_{x in X} f(x)
 *   Table 2          the reformulation   max_{x in X} max_{y in Y} F(x, y)
 *   Table 3          closed-form subproblems S1..S6 and their optimal values
 *   Section 2.1      operators T_s, U_gamma (eq. 5), V_gamma (eq. 6), lambda_s
 *   Algorithm 2      the AM loop; the stopping rule below it (Section 2.2)
 *   Section 4.1      the sparsity-targeting rule for gamma used in the paper's runs
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - sgn(0) = +1 in the y-step of the L1-variance forms, so y is in {-1,+1}^n;
 *   - T_s keeps, among equal |a_i|, the lower index;
 *   - U_gamma keeps a_i iff a_i^2 > gamma (strict; [sgn(0)]_+ = 0 in eq. 5);
 *   - x is normalised after every x-step (Section 2.2 recommends it numerically);
 *   - the stop test F_{k+1} <= (1 + tol) F_k is applied from the second sweep on
 *     (it needs two values), only between sweeps that use the same gamma, and never
 *     when tol < 0 (then exactly max_iter sweeps run);
 *   - a zero x-step result (or Ax = 0 for L2 variance) ends the start as "degenerate"
 *     with x = 0, which is feasible for every formulation;
 *   - gamma-targeting (Section 4.1): during the first C sweeps gamma is set so that
 *     exactly s entries survive (the (s+1)-th largest a_i^2 for U_gamma, |a_i| for
 *     V_gamma, or 0 if s >= p) and it is frozen from then on.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* formulation numbers follow Table 1 */
enum { F_L2_L0CON = 1, F_L1_L0CON = 2, F_L2_L1CON = 3, F_L1_L1CON = 4,
       F_L2_L0PEN = 5, F_L1_L0PEN = 6, F_L2_L1PEN = 7, F_L1_L1PEN = 8 };

/* per-start status codes */
enum { ST_MAXITER = 0, ST_CONVERGED = 1, ST_DEGENERATE = 2 };

/* The data matrix A (n x p), stored dense (row-major) or as compressed sparse rows: row i's
 * entries are val[k] at column col[k] for ptr[i] <= k < ptr[i+1], in ascending column order
 * and without repeated columns.  Storage changes only which terms of the two products of
 * Algorithm 2 are formed: the sparse loops skip the entries that are zero and otherwise add
 * the same products in the same order as the dense ones, so both give the same FP64 result. */
typedef struct {
    int64_t n, p;
    const double *A;                       /* dense, or NULL */
    const int64_t *ptr;                    /* sparse rows */
    const int32_t *col;
    const double *val;
} Mat;

/* u = A x: u_i = sum_j A_ij x_j, j ascending */
static void mat_Ax(const Mat *M, const double *x, double *u)
{
    for (int64_t i = 0; i < M->n; ++i) {
        double acc = 0.0;
        if (M->A) {
            for (int64_t j = 0; j < M->p; ++j) acc += M->A[i * M->p + j] * x[j];
        } else {
            for (int64_t k = M->ptr[i]; k < M->ptr[i + 1]; ++k) acc += M->val[k] * x[M->col[k]];
        }
        u[i] = acc;
    }
}

/* v = A^T y: v_j = sum_i A_ij y_i, i ascending */
static void mat_ATy(const Mat *M, const double *y, double *v)
{
    for (int64_t j = 0; j < M->p; ++j) v[j] = 0.0;
    for (int64_t i = 0; i < M->n; ++i) {
        if (M->A) {
            for (int64_t j = 0; j < M->p; ++j) v[j] += M->A[i * M->p + j] * y[i];
        } else {
            for (int64_t k = M->ptr[i]; k < M->ptr[i + 1]; ++k) v[M->col[k]] += M->val[k] * y[i];
        }
    }
}

static int is_l1_variance(int form) { return form % 2 == 0; }           /* forms 2,4,6,8 */
static int is_penalty(int form)     { return form >= 5; }                /* forms 5..8   */
static int uses_U(int form)         { return form == 5 || form == 6; }   /* L0 penalty   */
static int uses_V(int form)         { return form == 7 || form == 8; }   /* L1 penalty   */
static int uses_T(int form)         { return form == 1 || form == 2; }   /* L0 constraint*/

/* ------------------------------------------------------------------------------------ */
/* ordering helper: (key descending, index ascending)                                   */
/* ------------------------------------------------------------------------------------ */
typedef struct { double key; int64_t idx; } keyed;

static int cmp_desc_then_index(const void *pa, const void *pb)
{
    const keyed *a = (const keyed *)pa, *b = (const keyed *)pb;
    if (a->key > b->key) return -1;
    if (a->key < b->key) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

/* the j-th largest (1-based) of key[0..m-1]; 0 if j > m */
static double jth_largest(const double *key, int64_t m, int64_t j)
{
    if (j > m || j < 1) return 0.0;
    keyed *w = (keyed *)malloc((size_t)m * sizeof(keyed));
    for (int64_t i = 0; i < m; ++i) { w[i].key = key[i]; w[i].idx = i; }
    qsort(w, (size_t)m, sizeof(keyed), cmp_desc_then_index);
    double out = w[j - 1].key;
    free(w);
    return out;
}

/* ------------------------------------------------------------------------------------ */
/* Section 2.1 operators                                                                */
/* ------------------------------------------------------------------------------------ */

/* T_s(a): keep the s largest |a_i| (ties: lower index), zero the rest. */
void oracle_op_T(const double *a, int64_t m, int64_t s, double *z)
{
    keyed *w = (keyed *)malloc((size_t)m * sizeof(keyed));
    for (int64_t i = 0; i < m; ++i) { w[i].key = fabs(a[i]); w[i].idx = i; }
    qsort(w, (size_t)m, sizeof(keyed), cmp_desc_then_index);
    for (int64_t i = 0; i < m; ++i) z[i] = 0.0;
    for (int64_t t = 0; t < s && t < m; ++t) z[w[t].idx] = a[w[t].idx];
    free(w);
}

/* eq. (5): (U_gamma(a))_i = a_i [sgn(a_i^2 - gamma)]_+ */
void oracle_op_U(const double *a, int64_t m, double gamma, double *z)
{
    for (int64_t i = 0; i < m; ++i) z[i] = (a[i] * a[i] > gamma) ? a[i] : 0.0;
}

/* eq. (6): (V_gamma(a))_i = sgn(a_i) (|a_i| - gamma)_+ */
void oracle_op_V(const double *a, int64_t m, double gamma, double *z)
{
    for (int64_t i = 0; i < m; ++i) {
        double t = fabs(a[i]) - gamma;
        double sg = (a[i] > 0.0) ? 1.0 : ((a[i] < 0.0) ? -1.0 : 0.0);
        z[i] = (t > 0.0) ? sg * t : 0.0;
    }
}

/*
 * lambda_s(a) = argmin_{lambda >= 0} lambda sqrt(s) + ||V_lambda(a)||_2   (Section 2.1).
 *
 * g(lambda) = lambda sqrt(s) + ||V_lambda(a)||_2 is convex; on an interval between two
 * consecutive sorted magnitudes b_{k+1} <= lambda <= b_k the active set is the top k
 * entries, with S1 = sum of their |a|, S2 = sum of their a^2, so
 *   ||V_lambda||_1 = S1 - k lambda,   ||V_lambda||_2^2 = S2 - 2 lambda S1 + k lambda^2.
 * g'(lambda) = sqrt(s) - ||V_lambda||_1 / ||V_lambda||_2, whose sign is the sign of
 *   phi(lambda) = s ||V_lambda||_2^2 - ||V_lambda||_1^2,
 * non-decreasing in lambda.  If phi(0) >= 0 the minimiser is 0 (the L1 ball is not
 * binding).  Otherwise walk the breakpoints from the top, find the piece on which phi
 * changes sign, and solve phi = 0 there:
 *   k (k - s) lambda^2 - 2 (k - s) S1 lambda + (S1^2 - s S2) = 0,
 *   lambda = ( S1 - sqrt( s (k S2 - S1^2) / (k - s) ) ) / k   (the root with sum w > 0).
 */
double oracle_lambda_s(const double *a, int64_t m, double s)
{
    double *b = (double *)malloc((size_t)(m + 1) * sizeof(double));
    keyed *w = (keyed *)malloc((size_t)m * sizeof(keyed));
    for (int64_t i = 0; i < m; ++i) { w[i].key = fabs(a[i]); w[i].idx = i; }
    qsort(w, (size_t)m, sizeof(keyed), cmp_desc_then_index);
    for (int64_t i = 0; i < m; ++i) b[i] = w[i].key;
    b[m] = 0.0;
    free(w);

    double n1 = 0.0, n2 = 0.0;
    for (int64_t i = 0; i < m; ++i) { n1 += b[i]; n2 += b[i] * b[i]; }
    if (s * n2 - n1 * n1 >= 0.0) { free(b); return 0.0; }       /* phi(0) >= 0 */

    double S1 = 0.0, S2 = 0.0, lambda = 0.0;
    for (int64_t k = 1; k <= m; ++k) {
        S1 += b[k - 1];
        S2 += b[k - 1] * b[k - 1];
        double lo = b[k];                                        /* b_{k+1} (1-based) */
        double sum_w = S1 - (double)k * lo;
        double sum_w2 = S2 - 2.0 * lo * S1 + (double)k * lo * lo;
        double phi_lo = s * sum_w2 - sum_w * sum_w;
        if (phi_lo < 0.0) {                                      /* root in (b_{k+1}, b_k] */
            double kk = (double)k;
            if (kk <= s) { lambda = lo; break; }                 /* unreachable in exact arithmetic */
            double disc = s * (kk * S2 - S1 * S1) / (kk - s);
            if (disc < 0.0) disc = 0.0;
            lambda = (S1 - sqrt(disc)) / kk;
            if (lambda < lo) lambda = lo;
            if (lambda > b[k - 1]) lambda = b[k - 1];
            break;
        }
    }
    free(b);
    return lambda;
}

/* ------------------------------------------------------------------------------------ */
/* x-step (Algorithm 2, with the Table 3 value of the subproblem)                       */
/* ------------------------------------------------------------------------------------ */

/*
 * One x-step on v = A^T y.  Writes x (normalised, or 0), the value F(x, y) of Table 3
 * (S3..S6), the number of nonzeros, and the threshold used (gamma or lambda_s).
 *   calibrate != 0 (penalty forms only): gamma is first set by the Section 4.1 rule.
 * Returns 1 if the result is the zero vector (degenerate), else 0.
 */
int oracle_xstep(int form, const double *v, int64_t p, double s, double gamma, int calibrate,
                 double *x, double *F_out, int64_t *nnz_out, double *thr_out)
{
    double F = 0.0, thr = gamma;
    if (uses_T(form)) {                                          /* S3 */
        oracle_op_T(v, p, (int64_t)s, x);
        thr = 0.0;
    } else if (form == F_L2_L1CON || form == F_L1_L1CON) {      /* S4 */
        thr = oracle_lambda_s(v, p, s);
        oracle_op_V(v, p, thr, x);
    } else if (uses_U(form)) {                                   /* S5 */
        if (calibrate) {
            double *key = (double *)malloc((size_t)p * sizeof(double));
            for (int64_t i = 0; i < p; ++i) key[i] = v[i] * v[i];
            thr = jth_largest(key, p, (int64_t)s + 1);
            free(key);
        }
        oracle_op_U(v, p, thr, x);
    } else {                                                     /* S6 */
        if (calibrate) {
            double *key = (double *)malloc((size_t)p * sizeof(double));
            for (int64_t i = 0; i < p; ++i) key[i] = fabs(v[i]);
            thr = jth_largest(key, p, (int64_t)s + 1);
            free(key);
        }
        oracle_op_V(v, p, thr, x);
    }

    double sq = 0.0;
    int64_t nnz = 0;
    for (int64_t i = 0; i < p; ++i) { sq += x[i] * x[i]; nnz += (x[i] != 0.0); }
    double nrm = sqrt(sq);

    if (uses_T(form))       F = nrm;                                  /* ||T_s(a)||_2            */
    else if (uses_U(form))  F = sq - thr * (double)nnz;               /* ||U||_2^2 - g ||U||_0   */
    else if (uses_V(form))  F = nrm;                                  /* ||V_gamma(a)||_2        */
    else                    F = thr * sqrt(s) + nrm;                  /* lambda sqrt(s) + ||V||_2*/

    *F_out = F;
    *nnz_out = nnz;
    *thr_out = thr;
    if (nrm == 0.0) return 1;
    for (int64_t i = 0; i < p; ++i) x[i] /= nrm;
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Table 1 objective and explained variance                                             */
/* ------------------------------------------------------------------------------------ */

/* f(x) of Table 1 (gamma = the penalty used) and the explained variance of Section 4.1
 * (||Ax||_2^2 for L2 variance, ||Ax||_1 for L1 variance). */
static void objective_of(const Mat *M, int form, double gamma, const double *x, double *u,
                         double *f_out, double *ev_out)
{
    double l1 = 0.0, l2sq = 0.0, x0 = 0.0, x1 = 0.0;
    mat_Ax(M, x, u);
    for (int64_t i = 0; i < M->n; ++i) {
        l1 += fabs(u[i]);
        l2sq += u[i] * u[i];
    }
    for (int64_t j = 0; j < M->p; ++j) { x0 += (x[j] != 0.0); x1 += fabs(x[j]); }
    double l2 = sqrt(l2sq), f;
    switch (form) {
    case F_L2_L0CON: case F_L2_L1CON: f = l2; break;
    case F_L1_L0CON: case F_L1_L1CON: f = l1; break;
    case F_L2_L0PEN: f = l2sq - gamma * x0; break;
    case F_L1_L0PEN: f = l1 * l1 - gamma * x0; break;
    case F_L2_L1PEN: f = l2 - gamma * x1; break;
    default:         f = l1 - gamma * x1; break;                 /* F_L1_L1PEN */
    }
    *f_out = f;
    *ev_out = is_l1_variance(form) ? l1 : l2sq;
}

void oracle_objective(const double *A, int64_t n, int64_t p, int form, double gamma,
                      const double *x, double *f_out, double *ev_out)
{
    Mat M = {n, p, A, NULL, NULL, NULL};
    double *u = (double *)malloc((size_t)n * sizeof(double));
    objective_of(&M, form, gamma, x, u, f_out, ev_out);
    free(u);
}

/* the same for A in compressed sparse rows */
void oracle_objective_csr(const int64_t *ptr, const int32_t *col, const double *val, int64_t n,
                          int64_t p, int form, double gamma, const double *x, double *f_out,
                          double *ev_out)
{
    Mat M = {n, p, NULL, ptr, col, val};
    double *u = (double *)malloc((size_t)n * sizeof(double));
    objective_of(&M, form, gamma, x, u, f_out, ev_out);
    free(u);
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 2 for one start                                                            */
/* ------------------------------------------------------------------------------------ */

/*
 * Runs Algorithm 2 from the raw start g (x^(0) = g / ||g||_2).
 *   M       the data matrix (n x p)
 *   x       out: final x (p)
 *   F_hist  out, optional: F(x^(k), y^(k-1)) for k = 1..iters (max_iter entries, rest NaN)
 * Returns the status (ST_*); *iters = number of sweeps (y-step + x-step) performed.
 */
static int am_one_start(const Mat *M, int form, double s,
                        double gamma, int gamma_target, int calib, int max_iter, double tol,
                        const double *g, double *x, double *u, double *y, double *v,
                        double *F_hist, int *iters, double *gamma_used, double *F_last)
{
    const int64_t n = M->n, p = M->p;
    /* Algorithm 2: select initial point */
    double nrm = 0.0;
    for (int64_t j = 0; j < p; ++j) nrm += g[j] * g[j];
    nrm = sqrt(nrm);
    for (int64_t j = 0; j < p; ++j) x[j] = (nrm > 0.0) ? g[j] / nrm : 0.0;
    if (F_hist) for (int k = 0; k < max_iter; ++k) F_hist[k] = NAN;

    int penalty = is_penalty(form);
    int C = (penalty && gamma_target) ? calib : 0;
    double g_cur = gamma, F_prev = 0.0, F = 0.0;
    int status = ST_MAXITER, k;
    if (nrm == 0.0) { *iters = 0; *gamma_used = g_cur; *F_last = 0.0; return ST_DEGENERATE; }

    for (k = 1; k <= max_iter; ++k) {
        /* u = A x^(k-1) */
        mat_Ax(M, x, u);
        /* y-step: S2 (L1 variance) or S1 (L2 variance) */
        if (is_l1_variance(form)) {
            for (int64_t i = 0; i < n; ++i) y[i] = (u[i] >= 0.0) ? 1.0 : -1.0;
        } else {
            double un = 0.0;
            for (int64_t i = 0; i < n; ++i) un += u[i] * u[i];
            un = sqrt(un);
            if (un == 0.0) {
                for (int64_t j = 0; j < p; ++j) x[j] = 0.0;
                status = ST_DEGENERATE; F = 0.0; break;
            }
            for (int64_t i = 0; i < n; ++i) y[i] = u[i] / un;
        }
        /* v = A^T y */
        mat_ATy(M, y, v);
        /* x-step (S3..S6) */
        int64_t nnz;
        double thr;
        int calibrate = (k <= C);
        int zero = oracle_xstep(form, v, p, s, g_cur, calibrate, x, &F, &nnz, &thr);
        if (penalty) g_cur = thr;
        if (F_hist) F_hist[k - 1] = F;
        if (zero) { status = ST_DEGENERATE; break; }
        /* stopping rule (Section 2.2) */
        if (tol >= 0.0 && k >= 2 && k >= C + 1 && F <= (1.0 + tol) * F_prev) {
            status = ST_CONVERGED; break;
        }
        F_prev = F;
    }
    *iters = (k > max_iter) ? max_iter : k;
    *gamma_used = g_cur;
    *F_last = F;
    return status;
}

/*
 * oracle_solve: Algorithm 2 from r raw starts (G is r x p, one start per row), then the
 * Table 1 objective of every result, and the best start (largest objective; for the
 * gamma-targeting mode of the penalty forms the largest explained variance, since each
 * start then has its own gamma); ties go to the lower start index.
 *
 * Outputs (each r-long unless noted; any may be NULL except X):
 *   X (r x p)  final x per start         f, ev     objective and explained variance
 *   F          last F value              iters     sweeps performed
 *   status     ST_*                      gam       gamma used (penalty forms)
 *   F_hist (r x max_iter)                nthreads  OpenMP threads over starts (<=0: all)
 * Returns the best start index.
 */
static int solve_of(const Mat *M, int form, double s, double gamma, int gamma_target, int calib,
                    const double *G, int r, int max_iter, double tol, double *X, double *f,
                    double *ev, double *F, int *iters, int *status, double *gam, double *F_hist,
                    int nthreads)
{
    const int64_t n = M->n, p = M->p;
    double *f_loc = (double *)malloc((size_t)r * sizeof(double));
    double *ev_loc = (double *)malloc((size_t)r * sizeof(double));
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int c = 0; c < r; ++c) {
        double *u = (double *)malloc((size_t)n * sizeof(double));
        double *y = (double *)malloc((size_t)n * sizeof(double));
        double *v = (double *)malloc((size_t)p * sizeof(double));
        int it, st;
        double g_used, F_last;
        st = am_one_start(M, form, s, gamma, gamma_target, calib, max_iter, tol,
                          G + (int64_t)c * p, X + (int64_t)c * p, u, y, v,
                          F_hist ? F_hist + (int64_t)c * max_iter : NULL, &it, &g_used, &F_last);
        objective_of(M, form, g_used, X + (int64_t)c * p, u, &f_loc[c], &ev_loc[c]);
        if (iters) iters[c] = it;
        if (status) status[c] = st;
        if (gam) gam[c] = g_used;
        if (F) F[c] = F_last;
        free(u); free(y); free(v);
    }
    int use_ev = is_penalty(form) && gamma_target;
    int best = 0;
    for (int c = 1; c < r; ++c) {
        double a = use_ev ? ev_loc[c] : f_loc[c], b = use_ev ? ev_loc[best] : f_loc[best];
        if (a > b) best = c;
    }
    if (f) memcpy(f, f_loc, (size_t)r * sizeof(double));
    if (ev) memcpy(ev, ev_loc, (size_t)r * sizeof(double));
    free(f_loc); free(ev_loc);
    return best;
}

int oracle_solve(const double *A, int64_t n, int64_t p, int form, double s, double gamma,
                 int gamma_target, int calib, const double *G, int r, int max_iter,
                 double tol, double *X, double *f, double *ev, double *F, int *iters,
                 int *status, double *gam, double *F_hist, int nthreads)
{
    Mat M = {n, p, A, NULL, NULL, NULL};
    return solve_of(&M, form, s, gamma, gamma_target, calib, G, r, max_iter, tol, X, f, ev, F,
                    iters, status, gam, F_hist, nthreads);
}

/* the same for A in compressed sparse rows (ascending columns within a row, none repeated) */
int oracle_solve_csr(const int64_t *ptr, const int32_t *col, const double *val, int64_t n,
                     int64_t p, int form, double s, double gamma, int gamma_target, int calib,
                     const double *G, int r, int max_iter, double tol, double *X, double *f,
                     double *ev, double *F, int *iters, int *status, double *gam,
                     double *F_hist, int nthreads)
{
    Mat M = {n, p, NULL, ptr, col, val};
    return solve_of(&M, form, s, gamma, gamma_target, calib, G, r, max_iter, tol, X, f, ev, F,
                    iters, status, gam, F_hist, nthreads);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
