"""Pins for the oracle's whole AM iteration (Algorithm 2) against what the paper and the
mathematics fix: brute-force global optima on tiny inputs, the PCA reduction (s = p,
gamma = 0), closed forms (s = 1, rank-one spike), monotonicity (Section 1.2), the sandwich
F_k <= f(x^k) <= F_{k+1}, and the AM = GPower equivalence (Theorem 1) run through an
independent numpy implementation of GPower."""
import itertools

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from paper_1212_4137_gb300 import inputs as I


def _starts(p, r, seed):
    return I.raw_starts(p, r, seed)


# ------------------------------------------------------------------------------ brute force
def _sigma_max(M):
    return float(np.linalg.svd(M, compute_uv=False)[0]) if M.size else 0.0


def _opt_L2_L0con(A, s):
    return max(_sigma_max(A[:, list(S)]) for S in itertools.combinations(range(A.shape[1]), s))


def _opt_L2_L0pen(A, gamma):
    best = 0.0
    for k in range(1, A.shape[1] + 1):
        for S in itertools.combinations(range(A.shape[1]), k):
            best = max(best, _sigma_max(A[:, list(S)]) ** 2 - gamma * k)
    return best


def _signs(n):
    # y and -y give the same value for every L1-variance form: fix y_0 = +1
    for bits in itertools.product((1.0, -1.0), repeat=n - 1):
        yield np.array((1.0,) + bits)


def _phi_S3(a, s):
    return max(np.linalg.norm(a[list(S)]) for S in itertools.combinations(range(a.size), s))


def _phi_S4(a, s):
    # max a^T x over ||x||_2 <= 1, ||x||_1 <= sqrt(s): the dual min over lambda (library minimiser)
    g = lambda t: t * np.sqrt(s) + np.linalg.norm(np.maximum(np.abs(a) - t, 0))
    r = minimize_scalar(g, bounds=(0, np.abs(a).max()), method="bounded", options={"xatol": 1e-13})
    return min(r.fun, g(0.0))


def _phi_S5(a, gamma):
    best = 0.0
    for k in range(1, a.size + 1):
        for S in itertools.combinations(range(a.size), k):
            best = max(best, float(np.sum(a[list(S)] ** 2)) - gamma * k)
    return best


def _phi_S6(a, gamma):
    return float(np.linalg.norm(a - np.clip(a, -gamma, gamma)))


def _opt_L1_variance(A, phi):
    """max_x max_{y in {-1,1}^n} y^T A x  =  max_y max_x (A^T y)^T x  =  max_y phi(A^T y)."""
    return max(phi(A.T @ y) for y in _signs(A.shape[0]))


def _best(res):
    return res.f[res.best]


@pytest.mark.parametrize("seed", range(4))
def test_form1_best_of_starts_reaches_brute_force(oracle, seed):
    A = I.gaussian_matrix(6, 8, 10 + seed)
    for s in (1, 2, 3):
        res = oracle.solve(A, 1, _starts(8, 64, 20 + seed), s=s, max_iter=200, tol=0)
        opt = _opt_L2_L0con(A, s)
        assert res.f.max() <= opt * (1 + 1e-12)
        assert abs(_best(res) - opt) < 1e-9 * opt


@pytest.mark.parametrize("seed", range(3))
def test_form5_best_of_starts_reaches_brute_force(oracle, seed):
    A = I.gaussian_matrix(6, 8, 30 + seed)
    for gamma in (0.5, 2.0, 6.0):
        res = oracle.solve(A, 5, _starts(8, 64, 40 + seed), gamma=gamma, max_iter=200, tol=0)
        opt = _opt_L2_L0pen(A, gamma)
        assert res.f.max() <= opt + 1e-9
        assert abs(_best(res) - opt) < 1e-9 * max(1.0, opt)


@pytest.mark.parametrize("form,param,phi", [
    (2, 2, lambda a: _phi_S3(a, 2)),
    (4, 2.0, lambda a: _phi_S4(a, 2.0)),
    (6, 1.5, lambda a: _phi_S5(a, 1.5)),
    (8, 0.7, lambda a: _phi_S6(a, 0.7)),
])
@pytest.mark.parametrize("seed", range(2))
def test_L1_variance_forms_reach_sign_enumeration(oracle, form, param, phi, seed):
    A = I.gaussian_matrix(7, 6, 50 + seed)
    kw = dict(s=param) if form in (2, 4) else dict(gamma=param)
    res = oracle.solve(A, form, _starts(6, 64, 60 + seed), max_iter=200, tol=0, **kw)
    # for form 6 the joint maximum of (y^T A x)^2 - gamma ||x||_0 is max_x ||Ax||_1^2 - gamma ||x||_0
    opt = _opt_L1_variance(A, phi)
    assert res.f.max() <= opt * (1 + 1e-9) + 1e-9
    assert abs(_best(res) - opt) < 1e-7 * max(1.0, opt)


def _circle_opt(A, phi, grid=20000):
    """n = 2: max over unit y (a circle) of phi(A^T y), dense grid + local refinement."""
    th = np.linspace(0, 2 * np.pi, grid, endpoint=False)
    vals = np.array([phi(A.T @ np.array([np.cos(t), np.sin(t)])) for t in th])
    t0 = th[np.argmax(vals)]
    r = minimize_scalar(lambda t: -phi(A.T @ np.array([np.cos(t), np.sin(t)])),
                        bounds=(t0 - 2 * np.pi / grid, t0 + 2 * np.pi / grid), method="bounded",
                        options={"xatol": 1e-12})
    return max(vals.max(), -r.fun)


@pytest.mark.parametrize("form,param,phi", [
    (3, 2.0, lambda a: _phi_S4(a, 2.0)),
    (7, 0.8, lambda a: _phi_S6(a, 0.8)),
])
def test_L2_variance_L1_forms_reach_circle_search(oracle, form, param, phi):
    """For n = 2 the L2-variance problems are max over the unit circle of phi(A^T y)."""
    A = I.gaussian_matrix(2, 7, 70 + form)
    kw = dict(s=param) if form == 3 else dict(gamma=param)
    res = oracle.solve(A, form, _starts(7, 64, 80), max_iter=300, tol=0, **kw)
    opt = _circle_opt(A, phi)
    assert res.f.max() <= opt * (1 + 1e-9)
    assert abs(_best(res) - opt) < 1e-7 * opt


# --------------------------------------------------------------------------- PCA reduction
@pytest.mark.parametrize("form,kw", [(1, dict(s=12)), (3, dict(s=12.0)), (5, dict(gamma=0.0)),
                                     (7, dict(gamma=0.0))])
def test_pca_reduction(oracle, form, kw):
    """s = p or gamma = 0 recovers classical PCA: the leading right singular vector."""
    A = I.gaussian_matrix(9, 12, 90)
    U, S, Vt = np.linalg.svd(A)
    res = oracle.solve(A, form, _starts(12, 4, 91), max_iter=2000, tol=0, **kw)
    target = S[0] ** 2 if form == 5 else S[0]
    for c in range(4):
        assert abs(res.f[c] - target) < 1e-10 * target
        assert min(np.abs(res.X[c] - Vt[0]).max(), np.abs(res.X[c] + Vt[0]).max()) < 1e-6


def test_robust_pca_reduction(oracle):
    """s = p in the L1-variance L0 form is robust PCA max ||Ax||_1 over the unit ball
    = max over sign vectors of ||A^T y||_2."""
    A = I.gaussian_matrix(8, 5, 92)
    res = oracle.solve(A, 2, _starts(5, 64, 93), s=5, max_iter=200, tol=0)
    opt = max(np.linalg.norm(A.T @ y) for y in _signs(8))
    assert abs(_best(res) - opt) < 1e-10 * opt


# ----------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("form", [1, 2, 3, 4])
def test_s_equals_one(oracle, form):
    """s = 1: the feasible set's extreme points are +-e_j, so OPT = max_j ||a_j|| (L2 or L1)."""
    A = I.gaussian_matrix(10, 9, 94)
    res = oracle.solve(A, form, _starts(9, 64, 95), s=1, max_iter=100, tol=0)
    colnorm = np.abs(A).sum(0) if form % 2 == 0 else np.linalg.norm(A, axis=0)
    assert abs(_best(res) - colnorm.max()) < 1e-12 * colnorm.max()
    assert np.count_nonzero(res.X[res.best]) == 1


def test_rank_one_spike_recovered_in_one_sweep(oracle):
    """A = theta u v^T with ||v||_0 <= s: form 1 returns x = +-v and f = theta after one sweep."""
    rng = np.random.default_rng(5)
    n, p, s, theta = 30, 40, 4, 7.5
    u = rng.standard_normal(n); u /= np.linalg.norm(u)
    v = np.zeros(p); v[[3, 11, 20, 33]] = rng.standard_normal(4); v /= np.linalg.norm(v)
    A = theta * np.outer(u, v)
    res = oracle.solve(A, 1, _starts(p, 8, 96), s=s, max_iter=1, tol=-1)
    for c in range(8):
        assert min(np.abs(res.X[c] - v).max(), np.abs(res.X[c] + v).max()) < 1e-14
        assert abs(res.f[c] - theta) < 1e-13


# ------------------------------------------------------------------------------- invariants
@pytest.mark.parametrize("form,kw", [(1, dict(s=10)), (2, dict(s=10)), (3, dict(s=10.0)),
                                     (4, dict(s=10.0)), (5, dict(gamma=4.0)), (6, dict(gamma=50.0)),
                                     (7, dict(gamma=0.8)), (8, dict(gamma=8.0))])
def test_F_monotone(oracle, form, kw):
    """Section 1.2: the objective values along the iteration never decrease."""
    A = I.gaussian_matrix(40, 120, 97)
    res = oracle.solve(A, form, _starts(120, 16, 98), max_iter=60, tol=-1, **kw)
    for c in range(16):
        h = res.F_hist[c, :res.iters[c]]
        assert np.all(np.diff(h) >= -1e-12 * np.abs(h[1:])), (c, h)


@pytest.mark.parametrize("form", [5, 6, 7, 8])
def test_F_monotone_after_gamma_freeze(oracle, form):
    A = I.spiked_matrix(60, 200, I.spiked_thetas(60, 200), 8, 99, dtype=np.float64)
    res = oracle.solve(A, form, _starts(200, 16, 100), s=8, gamma_target=True, calib=5,
                       max_iter=40, tol=-1)
    for c in range(16):
        if res.status[c] == oracle.ST_DEGENERATE:
            continue
        h = res.F_hist[c, 4:res.iters[c]]          # from sweep C = 5 on gamma is frozen
        assert np.all(np.diff(h) >= -1e-12 * np.abs(h[1:])), (c, h)


@pytest.mark.parametrize("form", [1, 2, 3, 4])
def test_sandwich_constrained(oracle, form):
    """F(x^k, y^{k-1}) <= f(x^k) = max_y F(x^k, y) <= F(x^{k+1}, y^k)."""
    A = I.gaussian_matrix(30, 50, 101)
    G = _starts(50, 3, 102)
    K = 8
    full = oracle.solve(A, form, G, s=5, max_iter=K + 1, tol=-1)
    for k in range(1, K + 1):
        part = oracle.solve(A, form, G, s=5, max_iter=k, tol=-1)
        for c in range(3):
            fk = np.abs(A @ part.X[c]).sum() if form % 2 == 0 else np.linalg.norm(A @ part.X[c])
            assert full.F_hist[c, k - 1] <= fk * (1 + 1e-12)
            assert fk <= full.F_hist[c, k] * (1 + 1e-12)


# ----------------------------------------------------------------------- Theorem 1 (GPower)
def _gp_argmax_L0(g, s):
    idx = np.argsort(-np.abs(g), kind="stable")[:s]
    z = np.zeros_like(g); z[idx] = g[idx]
    return z / np.linalg.norm(z)


def _gp_argmax_L1ball(g, s):
    # maximiser over ||z||_2 <= 1, ||z||_1 <= sqrt(s): soft threshold at the lambda that
    # makes ||z||_1 = sqrt(s) ||z||_2, found here by plain bisection (not the oracle's method)
    if np.abs(g).sum() <= np.sqrt(s) * np.linalg.norm(g):
        return g / np.linalg.norm(g)
    lo, hi = 0.0, np.abs(g).max()
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        w = np.maximum(np.abs(g) - mid, 0)
        if np.sqrt(s) * np.linalg.norm(w) < w.sum():
            lo = mid
        else:
            hi = mid
    w = np.sign(g) * np.maximum(np.abs(g) - 0.5 * (lo + hi), 0)
    return w / np.linalg.norm(w)


def _gpower_constrained(A, form, x0, s, K):
    """Theorem 1, constrained forms: GPower on F_Y(x) over X; F_Y'(x) = A^T A x / ||Ax||_2
    (L2 variance) or A^T sgn(Ax) (L1 variance, sgn(0) = +1)."""
    x = x0 / np.linalg.norm(x0)
    out = []
    for _ in range(K):
        Ax = A @ x
        grad = A.T @ (np.where(Ax >= 0, 1.0, -1.0) if form % 2 == 0 else Ax / np.linalg.norm(Ax))
        x = _gp_argmax_L0(grad, int(s)) if form in (1, 2) else _gp_argmax_L1ball(grad, s)
        out.append(x)
    return out


def _gpower_penalized(A, form, y0, gamma, K):
    """Theorem 1, penalised forms: GPower on F_X(y) over Y.  F_X'(y) = 2 A U_gamma(A^T y)
    (L0 penalty) or A x(y) with x(y) = argmax_x F(x, y) (L1 penalty)."""
    y = y0
    out = []
    for _ in range(K):
        a = A.T @ y
        if form in (5, 6):
            z = np.where(a * a > gamma, a, 0.0)
            grad = 2 * A @ z
        else:
            w = np.sign(a) * np.maximum(np.abs(a) - gamma, 0)
            grad = A @ (w / np.linalg.norm(w))
        y = np.where(grad >= 0, 1.0, -1.0) if form % 2 == 0 else grad / np.linalg.norm(grad)
        out.append(y)
    return out


@pytest.mark.parametrize("form,param", [(1, 4), (2, 4), (3, 3.0), (4, 3.0)])
def test_theorem1_constrained_x_iterates(oracle, form, param):
    A = I.gaussian_matrix(20, 30, 103)
    G = _starts(30, 2, 104)
    K = 6
    for c in range(2):
        gp = _gpower_constrained(A, form, G[c], param, K)
        for k in range(1, K + 1):
            am = oracle.solve(A, form, G[c:c + 1], s=param, max_iter=k, tol=-1)
            assert np.abs(am.X[0] - gp[k - 1]).max() < 1e-9


@pytest.mark.parametrize("form,gamma", [(5, 0.6), (6, 20.0), (7, 0.3), (8, 3.0)])
def test_theorem1_penalized_y_iterates(oracle, form, gamma):
    A = I.gaussian_matrix(20, 30, 105)
    G = _starts(30, 2, 106)
    K = 6
    for c in range(2):
        x0 = G[c] / np.linalg.norm(G[c])
        Ax0 = A @ x0
        y0 = np.where(Ax0 >= 0, 1.0, -1.0) if form % 2 == 0 else Ax0 / np.linalg.norm(Ax0)
        gp = _gpower_penalized(A, form, y0, gamma, K)
        for k in range(1, K + 1):
            am = oracle.solve(A, form, G[c:c + 1], gamma=gamma, max_iter=k, tol=-1)
            Ax = A @ am.X[0]
            y_am = np.where(Ax >= 0, 1.0, -1.0) if form % 2 == 0 else Ax / np.linalg.norm(Ax)
            assert np.abs(y_am - gp[k - 1]).max() < 1e-9


# --------------------------------------------------------------------- stopping and edges
def test_stop_rule(oracle):
    A = I.gaussian_matrix(30, 60, 107)
    G = _starts(60, 4, 108)
    res = oracle.solve(A, 1, G, s=5, max_iter=500, tol=1e-9)
    assert np.all(res.status == oracle.ST_CONVERGED)
    for c in range(4):
        h = res.F_hist[c, :res.iters[c]]
        assert h[-1] <= (1 + 1e-9) * h[-2]
        assert np.all(h[1:-1] > (1 + 1e-9) * h[:-2])
    huge = oracle.solve(A, 1, G, s=5, max_iter=500, tol=1.0)
    assert np.all(huge.iters == 2)
    never = oracle.solve(A, 1, G, s=5, max_iter=37, tol=-1)
    assert np.all(never.iters == 37) and np.all(never.status == oracle.ST_MAXITER)


def test_degenerate_cases(oracle):
    A = I.gaussian_matrix(10, 20, 109)
    G = _starts(20, 3, 110)
    # gamma above every v_i^2: x = 0 after the first sweep, objective 0
    res = oracle.solve(A, 5, G, gamma=1e9, max_iter=10, tol=1e-9)
    assert np.all(res.status == oracle.ST_DEGENERATE) and np.all(res.iters == 1)
    assert not res.X.any() and np.all(res.f == 0.0)
    res = oracle.solve(A, 8, G, gamma=1e9, max_iter=10, tol=1e-9)
    assert np.all(res.status == oracle.ST_DEGENERATE)
    # A = 0: Ax = 0 in the L2 y-step
    res = oracle.solve(np.zeros((10, 20)), 1, G, s=3, max_iter=10, tol=1e-9)
    assert np.all(res.status == oracle.ST_DEGENERATE) and not res.X.any()
    # a zero start
    res = oracle.solve(A, 1, np.zeros((1, 20)), s=3, max_iter=10, tol=1e-9)
    assert res.status[0] == oracle.ST_DEGENERATE and res.iters[0] == 0


def test_best_start_ties_lowest_index(oracle):
    A = I.gaussian_matrix(10, 20, 111)
    g = _starts(20, 1, 112)
    res = oracle.solve(A, 1, np.repeat(g, 5, axis=0), s=3, max_iter=50, tol=1e-9)
    assert res.best == 0 and np.all(res.f == res.f[0])
