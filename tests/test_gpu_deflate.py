"""GPU parity of spca_deflate (projection deflation A <- A (I - z z^T), z = x / ||x||) against the
FP64 oracle's deflation, through the contractions of the deflated handle, and of a sequence of
components (solve, deflate by the best x, solve again) against the same sequence in FP64."""
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


def _products(lib, h, form, engine, X):
    import torch
    r, p = X.shape
    n = h.n
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    Ud = torch.zeros((r, n), dtype=torch.float32, device="cuda")
    Vd = torch.zeros((r, p), dtype=torch.float32, device="cuda")
    assert lib.spca_products(h.h, form, engine, Xd.data_ptr(), p, r, Ud.data_ptr(), n, Vd.data_ptr(), p) == 0
    torch.cuda.synchronize()
    return Ud.cpu().numpy().astype(np.float64), Vd.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("engine", ["simt", "tc"])
def test_deflated_products_match_fp64(lib, oracle, engine):
    n, p, r = 700, 1900, 48
    A = I.spiked_matrix(n, p, I.spiked_thetas(n, p), 20, 41, dtype=np.float32)
    rng = np.random.default_rng(42)
    x = rng.standard_normal(p).astype(np.float32) * 3.0          # not normalised
    D = oracle.deflate(A.astype(np.float64), x.astype(np.float64))
    X = rng.standard_normal((r, p)).astype(np.float32)
    X[1] = x                                                      # D z = 0
    eng = {"simt": lib.SPCA_ENGINE_SIMT, "tc": lib.SPCA_ENGINE_TC}[engine]
    h = lib.Handle(A)
    h.deflate(x)
    U, V = _products(lib, h, 1, eng, X)
    h.close()
    X64 = X.astype(np.float64)
    # the deflated FP32 entries are the FP64 ones rounded once (2^-24), the contraction adds its own
    scale_u = np.abs(X64) @ np.abs(D).T
    assert np.max(np.abs(U - X64 @ D.T) / (scale_u + 1e-300)) <= 2e-5
    assert np.max(np.abs(U[1])) <= 2e-5 * scale_u[1].max()
    Y = U / np.linalg.norm(U, axis=1, keepdims=True)
    scale_v = np.abs(Y) @ np.abs(D)
    assert np.max(np.abs(V - Y @ D) / (scale_v + 1e-300)) <= 2e-5


def test_three_components_match_fp64_sequence(lib, oracle):
    """Three well-separated sparse spikes: each solve (formulation 1, s = 20) finds one, and the
    deflation by its x makes the next solve find the next; the objective and support of every
    component match the FP64 sequence (oracle solve, oracle deflation by the oracle's x)."""
    n, p, s, r = 500, 1500, 20, 24
    A = I.spiked_matrix(n, p, I.spiked_thetas(n, p, base=(60.0, 40.0, 25.0)), 20, 43, dtype=np.float32)
    G = I.raw_starts(p, r, 44).astype(np.float32)
    h = lib.Handle(A)
    D64 = A.astype(np.float64)
    for comp in range(3):
        out = h.solve(1, r, s=float(s), x0=G, max_iter=200, tol=1e-9)
        ref = oracle.solve(D64, 1, G.astype(np.float64), s=float(s), max_iter=200, tol=1e-9)
        xr = ref.X[ref.best]
        assert abs(out["objective"] - ref.f[ref.best]) <= 1e-5 * ref.f[ref.best], (comp, out["objective"])
        assert np.array_equal(out["support"], np.flatnonzero(xr)), comp
        h.deflate(out["x"])
        D64 = oracle.deflate(D64, xr)
    h.close()


def test_deflate_rejects_bad_input(lib):
    A = I.gaussian_matrix(50, 80, 45).astype(np.float32)
    h = lib.Handle(A)
    with pytest.raises(lib.SpcaError) as e:
        h.deflate(np.zeros(80, np.float32))
    assert e.value.status == lib.SPCA_E_INVALID
    bad = np.ones(80, np.float32)
    bad[3] = np.nan
    with pytest.raises(lib.SpcaError) as e:
        h.deflate(bad)
    assert e.value.status == lib.SPCA_E_INVALID
    # the handle is unchanged and usable
    out = h.solve(1, 4, s=5.0, seed=3, max_iter=5, tol=-1)
    assert out["sweeps_total"] == 20
    h.close()
