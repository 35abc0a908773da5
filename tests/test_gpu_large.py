"""Parity on the large spiked configuration: n = 20000, p = 50000, 4096 starts, formulations 1 and
2 with s = 100, 20 sweeps on the 16-bit leading planes, then FP32 sweeps to the stopping rule
(tol 1e-9, at most 60 sweeps in all).  As at the benchmark's size, the FP64 oracle checks outputs it
can compute one by one, on 64 of the starts (the best one and 63 others): the Table 1 objective of the returned x; stationarity
(one FP64 sweep from a converged x gives it back, supports differing at most at the selection
threshold; a start that ran out of sweeps does not lose f to that sweep); feasibility; the best
start is the argmax; y of the best start is y(x) of the FP64 u = A x."""
import numpy as np
import pytest

from paper_1212_4137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N, P, R, S = 20000, 50000, 4096, 100


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
    A = I.spiked_matrix(N, P, I.spiked_thetas(N, P), 100, 20000, dtype=np.float32)
    h = lib.Handle(torch.from_numpy(A).cuda())
    yield A, h
    h.close()


def _near_threshold(A64, form, x, s, rel=1e-4):
    u = A64 @ x
    y = np.where(u >= 0, 1.0, -1.0) if form % 2 == 0 else u / np.linalg.norm(u)
    a = np.sort(np.abs(A64.T @ y))[::-1]
    k = int(s)
    t = [a[k - 1]] + ([a[k]] if a[k - 1] - a[k] <= rel * a[k - 1] else [])
    full = np.abs(A64.T @ y)
    near = np.zeros(full.size, bool)
    for tt in t:
        near |= np.abs(full - tt) <= rel * tt
    return near


@pytest.mark.parametrize("form", [1, 2])
def test_large_sampled_starts(lib, oracle, problem, form):
    A, h = problem
    out = h.solve(form, R, s=float(S), seed=20001, max_iter=60, tol=1e-9, lowp_sweeps=20, want_starts=True)
    X, f, status, iters = out["start_x"], out["start_objective"], out["start_status"], out["start_iters"]
    assert out["best_start"] == int(np.argmax(f))
    assert np.all(iters[status != lib.SPCA_ST_DEGENERATE] >= 22)   # 20 low-precision + 2 FP32
    A64 = A.astype(np.float64)
    # the FP64 oracle on 64 of the starts: the best one and 63 others
    rng = np.random.default_rng(20002 + form)
    others = [int(q) for q in rng.choice(np.delete(np.arange(R), out["best_start"]), 63, replace=False)]
    sample = [out["best_start"]] + others
    Xs = X[sample].astype(np.float64)
    for c, x in zip(sample, Xs):
        nz = np.flatnonzero(x)
        assert nz.size <= S and abs(np.linalg.norm(x) - 1.0) < 1e-5
    # objectives of the 64 x's in FP64 (the definition: ||Ax||_2, ||Ax||_1)
    Us = A64 @ Xs.T
    fo = np.linalg.norm(Us, axis=0) if form == 1 else np.abs(Us).sum(axis=0)
    assert np.all(np.abs(f[sample] - fo) <= 1e-9 * np.abs(fo)), np.max(np.abs(f[sample] - fo) / np.abs(fo))
    # one FP64 oracle sweep from each of the 64 x's (OpenMP over the starts)
    one = oracle.solve(A64, form, Xs, s=float(S), max_iter=1, tol=-1)
    for q, c in enumerate(sample):
        x = Xs[q]
        if status[c] == lib.SPCA_ST_CONVERGED:
            moved = (one.X[q] != 0) != (x != 0)
            if moved.any():
                assert np.all(_near_threshold(A64, form, x, S)[moved]), c
            else:
                assert np.max(np.abs(one.X[q] - x)) <= 1e-3, c
        else:
            fo1, _ = oracle.objective(A64, form, 0.0, one.X[q])
            assert fo1 >= fo[q] - 1e-6 * abs(fo[q]), (c, fo1, fo[q])
    b = out["best_start"]
    u = A64 @ X[b].astype(np.float64)
    y = out["y"].astype(np.float64)
    if form == 2:
        clear = np.abs(u) > 1e-6 * np.abs(u).max()
        assert np.array_equal(y[clear], np.where(u[clear] >= 0, 1.0, -1.0))
    else:
        assert np.max(np.abs(y - u / np.linalg.norm(u))) <= 1e-5
