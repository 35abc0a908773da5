"""Parity on the large spiked configuration: n = 20000, p = 50000, 4096 starts, formulations 1 and
2 with s = 100, 20 sweeps on the 16-bit leading planes, then FP32 sweeps to the stopping rule
(tol 1e-9, at most 60 sweeps in all).  As at the benchmark's size, the FP64 oracle checks outputs it
can compute one by one on sampled starts: the Table 1 objective of the returned x; stationarity
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
    rng = np.random.default_rng(20002 + form)
    for c in [out["best_start"]] + [int(q) for q in rng.choice(R, 5, replace=False)]:
        x = X[c].astype(np.float64)
        nz = np.flatnonzero(x)
        assert nz.size <= S and abs(np.linalg.norm(x) - 1.0) < 1e-5
        fo, _ = oracle.objective(A64, form, 0.0, x)
        assert abs(f[c] - fo) <= 1e-9 * abs(fo), (c, f[c], fo)
        one = oracle.solve(A64, form, x[None, :], s=float(S), max_iter=1, tol=-1)
        if status[c] == lib.SPCA_ST_CONVERGED:
            moved = (one.X[0] != 0) != (x != 0)
            if moved.any():
                assert np.all(_near_threshold(A64, form, x, S)[moved]), c
            else:
                assert np.max(np.abs(one.X[0] - x)) <= 1e-3, c
        else:
            fo1, _ = oracle.objective(A64, form, 0.0, one.X[0])
            assert fo1 >= fo - 1e-6 * abs(fo), (c, fo1, fo)
    b = out["best_start"]
    u = A64 @ X[b].astype(np.float64)
    y = out["y"].astype(np.float64)
    if form == 2:
        clear = np.abs(u) > 1e-6 * np.abs(u).max()
        assert np.array_equal(y[clear], np.where(u[clear] >= 0, 1.0, -1.0))
    else:
        assert np.max(np.abs(y - u / np.linalg.norm(u))) <= 1e-5
