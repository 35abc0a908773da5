"""Parity at the benchmark's full size, in the configuration bench.py times: the spiked model
n = 5000, p = 20000 with 1024 starts, all 8 formulations (s = 50, the Section 4.1 gamma rule for
the penalties, at most 100 sweeps, tol 1e-9).  The FP64 oracle cannot run 1024 starts for 100
sweeps here, so the test checks outputs it can compute one by one, on a sample of starts per
formulation (the best one and seven others):

- the Table 1 objective and the explained variance of each sampled start's x, recomputed in FP64;
- stationarity: one oracle sweep from a converged start's x (with that start's final gamma)
  gives x back, unless the supports differ only in entries whose |v_i| lies within 1e-4 of the
  selection threshold (the s-th largest |v_i|, lambda_s, sqrt(gamma) or gamma), where FP32 and
  FP64 may legitimately decide differently; starts that ran out of sweeps must not lose f to
  that sweep (Algorithm 2 is monotone);
- feasibility: unit norm, at most s nonzeros (L0 constraint), L1 norm at most sqrt(s) (L1
  constraint), and the support list equals the nonzeros of x;
- the best start is the argmax of the per-start objectives (explained variances in the
  gamma-targeting mode), ties to the lower index;
- y of the best start is y(x) of Table 3 (S2 or S1) of the FP64 u = A x."""
import numpy as np
import pytest

import bench
from paper_1212_4137_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _f_scale(form, ref):
    """Magnitude of the terms of the sweep's Table 3 value, the scale of its rounding error: the
    penalty values are differences, S5 = sum_S v_i^2 - gamma |S| and S6 = x^T v - gamma ||x||_1
    (x = V_gamma(v) / ||V_gamma(v)||_2), so a relative error eps in v moves them by about eps
    times |F| + gamma |S| or |F| + gamma ||x||_1."""
    F, x, g = abs(ref.F[0]), ref.X[0], ref.gamma[0]
    if form in (5, 6):
        return F + g * np.count_nonzero(x)
    if form in (7, 8):
        return F + g * np.abs(x).sum()
    return F

W = bench.WORKLOADS["spiked-5000x20000-r1024"]


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1212_4137_gb300 import build, spca
    build.build()
    spca.load()
    return spca


@pytest.fixture(scope="module")
def problem(lib):
    import torch
    A = bench.make_inputs(W)
    G = I.raw_starts(W["p"], W["r"], W["start_seed"]).astype(np.float32)
    h = lib.Handle(torch.from_numpy(A).cuda())
    yield A, A.astype(np.float64), G, h
    h.close()


def _near_threshold(oracle, A64, form, x, s, gamma, rel=1e-4):
    """Entries whose |v_i|, v = A^T y(x) in FP64, lie within rel of the x-step's threshold."""
    u = A64 @ x
    y = np.where(u >= 0, 1.0, -1.0) if form % 2 == 0 else u / np.linalg.norm(u)
    a = np.abs(A64.T @ y)
    if form in (1, 2):
        srt = np.sort(a)[::-1]
        k = int(s)
        t = [srt[k - 1]] + ([srt[k]] if k < a.size and srt[k - 1] - srt[k] <= rel * srt[k - 1] else [])
    elif form in (3, 4):
        t = [oracle.lambda_s(a, s)]
    elif form in (5, 6):
        t = [np.sqrt(gamma)]
    else:
        t = [gamma]
    near = np.zeros(a.size, bool)
    for tt in t:
        if tt > 0:
            near |= np.abs(a - tt) <= rel * tt
    return near


@pytest.mark.parametrize("form", range(1, 9))
def test_fullsize_sampled_starts(lib, oracle, problem, form):
    A, A64, G, h = problem
    r, s = W["r"], float(W["s"])
    kw = bench.solve_kwargs(W, form)
    out = h.solve(form, r, max_iter=W["max_iter"], tol=W["tol"], x0=G, want_starts=True, **kw)
    X, f, ev = out["start_x"], out["start_objective"], out["start_explained"]
    status, gam, iters = out["start_status"], out["start_gamma"], out["start_iters"]
    target = form >= 5

    # best start: argmax with ties to the lower index
    key = ev if target else f
    assert out["best_start"] == int(np.argmax(key))
    assert out["objective"] == f[out["best_start"]]

    rng = np.random.default_rng(100 + form)
    sample = [out["best_start"]] + [int(c) for c in rng.choice(r, 7, replace=False)]
    for c in sample:
        x = X[c].astype(np.float64)
        nz = np.flatnonzero(x)
        if status[c] == lib.SPCA_ST_DEGENERATE:
            assert nz.size == 0
            continue
        assert abs(np.linalg.norm(x) - 1.0) < 1e-5
        if form in (1, 2):
            assert nz.size <= s
        if form in (3, 4):
            assert np.abs(x).sum() <= np.sqrt(s) * (1 + 1e-5)
        # objective and explained variance of this x in FP64 (the start's final gamma)
        fo, evo = oracle.objective(A64, form, gam[c], x)
        assert abs(f[c] - fo) <= 1e-9 * max(1.0, abs(fo)), (c, f[c], fo)
        assert abs(ev[c] - evo) <= 1e-9 * max(1.0, abs(evo)), (c, ev[c], evo)
        # one FP64 sweep of the method from x, with the start's gamma frozen
        okw = dict(s=s) if form <= 4 else dict(s=s, gamma=gam[c])
        one = oracle.solve(A64, form, x[None, :], max_iter=1, tol=-1, **okw)
        step = np.max(np.abs(one.X[0] - x))
        if status[c] == lib.SPCA_ST_CONVERGED:
            moved = (one.X[0] != 0) != (x != 0)
            if moved.any():
                near = _near_threshold(oracle, A64, form, x, s, gam[c])
                assert np.all(near[moved]), (c, np.flatnonzero(moved & ~near)[:5])
            else:
                assert step <= 1e-3, (c, step)
        else:
            assert status[c] == lib.SPCA_ST_MAXITER and iters[c] == W["max_iter"]
            fo1, evo1 = oracle.objective(A64, form, gam[c], one.X[0])
            assert fo1 >= fo - 1e-6 * abs(fo), (c, fo1, fo)

    # y of the best start against S2 / S1 of the FP64 u = A x
    b = out["best_start"]
    u = A64 @ X[b].astype(np.float64)
    y = out["y"].astype(np.float64)
    if form % 2 == 0:
        clear = np.abs(u) > 1e-6 * np.abs(u).max()
        assert np.array_equal(y[clear], np.where(u[clear] >= 0, 1.0, -1.0))
    else:
        assert np.max(np.abs(y - u / np.linalg.norm(u))) <= 1e-5
    # the support list is the nonzeros of the best x
    assert np.array_equal(out["support"], np.flatnonzero(X[b]))


def _near_tie(A64, form, xk, s, gamma, gap=1e-4):
    """True if this sweep's hard selection (top-s for T_s and the gamma-targeting rule, v_i^2 >
    gamma for a frozen gamma) has its boundary within `gap` (relative) in the FP64 v."""
    if form in (3, 4, 7, 8):
        return False                       # soft thresholds are continuous in v
    u = A64 @ xk
    y = np.where(u >= 0, 1.0, -1.0) if form % 2 == 0 else u / np.linalg.norm(u)
    a = np.sort(np.abs(A64.T @ y))[::-1]
    if gamma is not None:
        return bool(np.min(np.abs(a * a - gamma)) <= gap * gamma)
    return bool((a[s - 1] - a[s]) <= gap * a[s - 1])


@pytest.mark.parametrize("form", range(1, 9))
def test_fullsize_single_sweep_parity(lib, oracle, problem, form):
    """One sweep of the GPU from its own iterate x^(k) at the benchmark's size and launch
    configuration (1024 starts: the CTA-pair contraction with 76 stream-K slots over 79 x 4
    tiles and K = 5000, the 1024-start support gather and candidate filter) against one FP64
    oracle sweep from the same x^(k), k in {1, 2, 5, 30}, on 16 sampled starts per k.  Early
    sweeps (k = 1, 2) are where the threshold still falls faster than the candidate guesses
    allow, so starts there also take the full x-step pass.  Bars: F within 1e-5 relative (the
    L0-penalty value scaled by its terms), x within 1e-4 in the infinity norm, and identical
    supports for the hard selections (forms 1, 2, 5, 6) unless the selection boundary lies within
    1e-4 of a tie in the FP64 v."""
    A, A64, G, h = problem
    r, s, C = W["r"], int(W["s"]), W["calib"]
    kw = bench.solve_kwargs(W, form)
    rng = np.random.default_rng(300 + form)
    checked = total = 0
    for k in (1, 2, 5, 30):
        o = h.solve(form, r, max_iter=k, tol=-1, x0=G, want_starts=True, **kw)
        o1 = h.solve(form, r, max_iter=k + 1, tol=-1, x0=G, want_starts=True, **kw)
        Xk, stat = o["start_x"].astype(np.float64), o["start_status"]
        for c in sorted(int(q) for q in rng.choice(r, 16, replace=False)):
            if stat[c] == lib.SPCA_ST_DEGENERATE or o1["start_status"][c] == lib.SPCA_ST_DEGENERATE:
                continue
            total += 1
            if form <= 4:
                okw = dict(s=float(s))
            elif k + 1 > C:                 # gamma frozen after the calibration sweeps
                okw = dict(gamma=float(o1["start_gamma"][c]))
            else:                           # this sweep re-targets gamma (Section 4.1)
                okw = dict(s=float(s), gamma_target=True, calib=1)
            ref = oracle.solve(A64, form, Xk[c:c + 1], max_iter=1, tol=-1, **okw)
            fixed_gamma = okw["gamma"] if (form >= 5 and not okw.get("gamma_target")) else None
            if _near_tie(A64, form, Xk[c], s, fixed_gamma):
                continue
            scaleF = _f_scale(form, ref)
            assert abs(o1["start_F"][c] - ref.F[0]) <= 1e-5 * max(1.0, scaleF), (k, c, o1["start_F"][c], ref.F[0])
            err = np.abs(o1["start_x"][c] - ref.X[0]).max()
            assert err <= 1e-4, (form, k, c, err)
            if form in (1, 2, 5, 6):
                assert np.array_equal(o1["start_x"][c] != 0, ref.X[0] != 0), (k, c)
            checked += 1
    assert total >= 48 and checked >= 0.8 * total, (checked, total)
