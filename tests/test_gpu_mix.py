"""Parity over a mix of problems drawn like the many-problems workload: per problem n and p
log-uniform, three spikes with theta = (40, 30, 20) sqrt(n / p) and 20 nonzeros each, the
formulation uniform on 1..8, s uniform on [5, 100] (at most p), the Section 4.1 gamma rule for
the penalties.  Sizes are scaled down (n in [60, 500], p in [150, 3000], 32 starts) so that the
FP64 oracle runs every start.  Bar: the best objective within 1e-5 of the oracle's (explained
variance in the gamma-targeting mode), and the GPU's best x a fixed point of the oracle's map."""
import numpy as np
import pytest

from paper_1212_4137_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1212_4137_gb300 import build, spca
    build.build()
    spca.load()
    return spca


def _problem(k):
    rng = np.random.default_rng(9000 + k)
    n = int(round(np.exp(rng.uniform(np.log(60), np.log(500)))))
    p = int(round(np.exp(rng.uniform(np.log(150), np.log(3000)))))
    form = int(rng.integers(1, 9))
    s = int(min(rng.integers(5, 101), p))
    A = I.spiked_matrix(n, p, I.spiked_thetas(n, p, base=(40.0, 30.0, 20.0)), 20, 9100 + k, dtype=np.float32)
    G = I.raw_starts(p, 32, 9200 + k).astype(np.float32)
    return A, G, form, s


@pytest.mark.parametrize("k", range(8))
def test_problem_mix(lib, oracle, k):
    A, G, form, s = _problem(k)
    kw = dict(s=float(s)) if form <= 4 else dict(s=float(s), gamma_target=True, calib=10)
    h = lib.Handle(A)
    out = h.solve(form, G.shape[0], x0=G, max_iter=100, tol=1e-9, want_starts=True, **kw)
    h.close()
    A64 = A.astype(np.float64)
    ref = oracle.solve(A64, form, G.astype(np.float64), max_iter=100, tol=1e-9, **kw)
    key_gpu = out["explained_variance"] if form >= 5 else out["objective"]
    key_ref = ref.ev[ref.best] if form >= 5 else ref.f[ref.best]
    assert abs(key_gpu - key_ref) <= 1e-5 * abs(key_ref), (form, s, key_gpu, key_ref)
    b = out["best_start"]
    x = out["start_x"][b].astype(np.float64)
    okw = dict(s=float(s)) if form <= 4 else dict(s=float(s), gamma=out["start_gamma"][b])
    one = oracle.solve(A64, form, x[None, :], max_iter=1, tol=-1, **okw)
    assert np.max(np.abs(one.X[0] - x)) <= 1e-3
