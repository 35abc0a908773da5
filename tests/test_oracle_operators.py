"""Pins for the oracle's subproblem operators (Section 2.1, Table 3), against values the
paper prints and against brute force / library optimisation that shares nothing with the
oracle's own arithmetic."""
import itertools
import os

import numpy as np
import pytest
from scipy.optimize import minimize, minimize_scalar

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = np.array([float(t) for t in v.split()])
    return out


def test_Ts_worked_example(oracle):
    g = _read_golden("ts_worked_example.txt")
    np.testing.assert_array_equal(oracle.op_T(g["a"], int(g["s"][0])), g["Ts"])


def _brute_S3(a, s):
    """max a^T z over ||z||_2 <= 1, ||z||_0 <= s  =  max over supports |S| <= s of ||a_S||_2."""
    best = 0.0
    for k in range(1, s + 1):
        for S in itertools.combinations(range(a.size), k):
            best = max(best, float(np.sqrt(np.sum(a[list(S)] ** 2))))
    return best


@pytest.mark.parametrize("seed", range(6))
def test_S3_value_matches_brute_force(oracle, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(9)
    for s in (1, 2, 4, 9):
        xs = oracle.xstep(1, a, s)
        assert xs.nnz <= s
        assert abs(np.linalg.norm(xs.x) - 1.0) < 1e-14
        # the maximiser attains the optimum, which brute force over supports confirms
        assert abs(a @ xs.x - _brute_S3(a, s)) < 1e-12
        assert abs(xs.F - _brute_S3(a, s)) < 1e-12


def test_Ts_ties_keep_lower_index(oracle):
    a = np.array([1.0, -3.0, 3.0, 2.0, -3.0])
    np.testing.assert_array_equal(oracle.op_T(a, 2), [0, -3.0, 3.0, 0, 0])
    np.testing.assert_array_equal(oracle.op_T(a, 3), [0, -3.0, 3.0, 0, -3.0])


def _brute_S5(a, gamma):
    """max (a^T z)^2 - gamma ||z||_0 over ||z||_2 <= 1 = max over supports S (incl. the
    empty one) of ||a_S||^2 - gamma |S|."""
    best = 0.0
    for k in range(1, a.size + 1):
        for S in itertools.combinations(range(a.size), k):
            best = max(best, float(np.sum(a[list(S)] ** 2)) - gamma * k)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_S5_value_matches_brute_force(oracle, seed):
    rng = np.random.default_rng(100 + seed)
    a = rng.standard_normal(8) * 2
    for gamma in (0.0, 0.3, 1.0, 2.5, 50.0):
        xs = oracle.xstep(5, a, 1, gamma)
        ref = _brute_S5(a, gamma)
        assert abs(xs.F - ref) < 1e-12
        if ref > 0:
            assert abs((a @ xs.x) ** 2 - gamma * np.count_nonzero(xs.x) - ref) < 1e-12
        else:
            assert xs.degenerate and not xs.x.any()


@pytest.mark.parametrize("seed", range(6))
def test_S6_value_is_distance_to_box(oracle, seed):
    """max a^T z - gamma ||z||_1 over the unit ball equals min over ||w||_inf <= gamma of
    ||a - w||_2 (minimax), i.e. the distance from a to the box [-gamma, gamma]^m."""
    rng = np.random.default_rng(200 + seed)
    a = rng.standard_normal(11) * 3
    for gamma in (0.0, 0.5, 1.7, 100.0):
        xs = oracle.xstep(7, a, 1, gamma)
        dist = float(np.linalg.norm(a - np.clip(a, -gamma, gamma)))
        assert abs(xs.F - dist) < 1e-12
        if dist > 0:
            assert abs(a @ xs.x - gamma * np.abs(xs.x).sum() - dist) < 1e-12
            # no random feasible point does better
            Z = rng.standard_normal((2000, a.size))
            Z /= np.linalg.norm(Z, axis=1, keepdims=True)
            assert np.max(Z @ a - gamma * np.abs(Z).sum(1)) <= dist + 1e-12


def _g(a, s, lam):
    w = np.maximum(np.abs(a) - lam, 0.0)
    return lam * np.sqrt(s) + np.linalg.norm(w)


@pytest.mark.parametrize("seed", range(10))
def test_lambda_s_minimises_dual(oracle, seed):
    """lambda_s(a) = argmin_{lambda>=0} lambda sqrt(s) + ||V_lambda(a)||_2 (Section 2.1),
    checked with a bounded scalar minimiser of the definition."""
    rng = np.random.default_rng(300 + seed)
    a = rng.standard_normal(25) * (1 + seed)
    for s in (1.0, 2.0, 3.5, 10.0, 25.0):
        lam = oracle.lambda_s(a, s)
        res = minimize_scalar(lambda t: _g(a, s, t), bounds=(0, np.abs(a).max()), method="bounded",
                              options={"xatol": 1e-12})
        assert _g(a, s, lam) <= res.fun + 1e-10
        if lam > 0:
            # the optimum is interior: the dual objective does not improve nearby
            for d in (1e-6, -1e-6):
                assert _g(a, s, lam) <= _g(a, s, max(0.0, lam + d)) + 1e-12


def test_lambda_s_zero_when_l1_ball_inactive(oracle):
    a = np.array([3.0, 0.1, 0.0, -0.1])
    # ||a||_1 = 3.2 <= sqrt(2) ||a||_2  ->  lambda = 0, x = a / ||a||
    assert oracle.lambda_s(a, 2.0) == 0.0
    xs = oracle.xstep(3, a, 2.0)
    np.testing.assert_allclose(xs.x, a / np.linalg.norm(a), rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_S4_matches_constrained_solver(oracle, seed):
    """max a^T z s.t. ||z||_2 <= 1, ||z||_1 <= sqrt(s): the x-step's value and maximiser
    against SLSQP on the split form z = z+ - z- (many random restarts)."""
    rng = np.random.default_rng(400 + seed)
    m = 7
    a = rng.standard_normal(m)
    for s in (1.0, 2.0, 3.0, 5.0):
        xs = oracle.xstep(3, a, s)
        x = xs.x
        assert np.linalg.norm(x) <= 1 + 1e-12 and np.abs(x).sum() <= np.sqrt(s) + 1e-10
        assert abs(a @ x - xs.F) < 1e-10
        cons = [{"type": "ineq", "fun": lambda w: 1.0 - np.sum((w[:m] - w[m:]) ** 2)},
                {"type": "ineq", "fun": lambda w: np.sqrt(s) - np.sum(w)}]
        best = -np.inf
        for _ in range(20):
            w0 = np.abs(rng.standard_normal(2 * m)) * 0.1
            r = minimize(lambda w: -(a @ (w[:m] - w[m:])), w0, method="SLSQP",
                         bounds=[(0, None)] * (2 * m), constraints=cons,
                         options={"ftol": 1e-14, "maxiter": 500})
            if r.success:
                best = max(best, -r.fun)
        assert abs(best - xs.F) < 1e-7


def test_S1_S2_y_step_values(oracle):
    """For s = p the L0-constrained x-step is S1 (a / ||a||); for gamma = 0 U_gamma keeps
    every nonzero entry; V_0 is the identity."""
    a = np.array([0.5, -2.0, 0.0, 1.0])
    np.testing.assert_allclose(oracle.xstep(1, a, 4).x, a / np.linalg.norm(a), atol=1e-16)
    np.testing.assert_allclose(oracle.xstep(5, a, 1, 0.0).x, a / np.linalg.norm(a), atol=1e-16)
    np.testing.assert_allclose(oracle.xstep(7, a, 1, 0.0).x, a / np.linalg.norm(a), atol=1e-16)


def test_gamma_targeting_keeps_exactly_s(oracle):
    """Section 4.1: gamma chosen so that exactly s entries survive (distinct magnitudes)."""
    rng = np.random.default_rng(7)
    v = rng.standard_normal(40)
    for form in (5, 6, 7, 8):
        for s in (1, 5, 17, 39):
            xs = oracle.xstep(form, v, s, 0.0, calibrate=True)
            assert xs.nnz == s
            keep = np.argsort(-np.abs(v), kind="stable")[:s]
            assert set(np.flatnonzero(xs.x)) == set(keep)
        xs = oracle.xstep(form, v, 40, 0.0, calibrate=True)   # s >= p: gamma = 0
        assert xs.nnz == 40 and xs.thr == 0.0
