"""GPU checks of the solve options around Algorithm 2: low-precision sweeps (A rounded to 11
significant bits, the leading FP16 plane, or to 4 with FP8 E4M3 storage, for the first sweeps,
then FP32 sweeps to the stopping rule), the cap on the FP32 sweeps, the wall-clock limit, 16- and
8-bit storage handles, and the low-precision contractions themselves against FP64 with the bound
their rounding gives.

Low-precision sweeps change the trajectory, so a start may reach another stationary point than in
a plain FP32 solve, and in the gamma-targeting mode gamma is calibrated on the rounded v.  What
the FP32 refinement guarantees, and what is checked: no start stops before two FP32 sweeps; every
start's reported objective is the FP64 objective of its x; the best x is a fixed point of the
FP64 map (constrained forms); and, for L2 variance with a cardinality bound, a start that ends on
the same support as in the plain FP32 solve has the same objective."""
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


@pytest.fixture(scope="module")
def spiked():
    n, p = 700, 2600
    A = I.spiked_matrix(n, p, I.spiked_thetas(n, p), 20, 711, dtype=np.float32)
    G = I.raw_starts(p, 96, 712).astype(np.float32)
    return A, G


def _kw(form):
    if form in (1, 2, 3, 4):
        return dict(s=20.0)
    return dict(s=20.0, gamma_target=True, calib=8)


@pytest.mark.parametrize("storage", ["f32", "fp8"])
@pytest.mark.parametrize("form", range(1, 9))
def test_lowp_then_fp32_refines(lib, oracle, spiked, form, storage):
    A, G = spiked
    A64 = A.astype(np.float64)
    h = lib.Handle(A, storage=lib.SPCA_FP8_E4M3_COLSCALED if storage == "fp8" else lib.SPCA_F32)
    r = G.shape[0]
    ref = h.solve(form, r, x0=G, max_iter=80, tol=1e-7, want_starts=True, **_kw(form))
    got = h.solve(form, r, x0=G, max_iter=80, tol=1e-7, want_starts=True, lowp_sweeps=12, **_kw(form))
    h.close()
    # no start stops during the low-precision sweeps or on the first FP32 sweep
    done = got["start_status"] != lib.SPCA_ST_DEGENERATE
    assert np.all(got["start_iters"][done] >= 14)
    # reported objectives are the FP64 objectives of the returned x
    for c in range(0, r, 12):
        fo, evo = oracle.objective(A64, form, got["start_gamma"][c], got["start_x"][c].astype(np.float64))
        assert abs(got["start_objective"][c] - fo) <= 1e-9 * max(1.0, abs(fo))
    if form > 4:
        return
    # the best x is a fixed point of the FP64 map
    b = got["best_start"]
    x = got["start_x"][b].astype(np.float64)
    one = oracle.solve(A64, form, x[None, :], max_iter=1, tol=-1, s=20.0)
    if np.array_equal(one.X[0] != 0, x != 0):
        assert np.max(np.abs(one.X[0] - x)) <= 1e-3
    if form != 1:
        return
    # L2 variance with a cardinality bound: on a fixed support the fixed point is the leading
    # singular vector of A restricted to it, so a start that ends on the same support as in the
    # plain FP32 solve has the same objective
    same = [c for c in range(r) if np.array_equal(got["start_x"][c] != 0, ref["start_x"][c] != 0)
            and got["start_status"][c] == lib.SPCA_ST_CONVERGED and ref["start_status"][c] == lib.SPCA_ST_CONVERGED]
    assert len(same) >= 1
    for c in same:
        assert abs(got["start_objective"][c] - ref["start_objective"][c]) <= 1e-5 * abs(ref["start_objective"][c])


def test_refine_sweeps_cap(lib, spiked):
    A, G = spiked
    h = lib.Handle(A)
    out = h.solve(1, 32, x0=G[:32], s=20.0, max_iter=100, tol=-1, lowp_sweeps=5, refine_sweeps=3,
                  want_starts=True)
    h.close()
    assert np.all(out["start_iters"] == 8)
    assert out["sweeps_total"] == 8 * 32


def test_timeout_returns_status(lib, spiked):
    A, G = spiked
    h = lib.Handle(A)
    with pytest.raises(lib.SpcaError) as e:
        h.solve(1, 32, x0=G[:32], s=20.0, max_iter=10000, tol=-1, timeout_us=1)
    assert e.value.status == lib.SPCA_E_TIMEOUT
    # the handle stays usable
    out = h.solve(1, 32, x0=G[:32], s=20.0, max_iter=5, tol=-1)
    assert out["sweeps_total"] == 5 * 32
    h.close()


def test_lowp_needs_tensor_cores_engine(lib, spiked):
    A, G = spiked
    h = lib.Handle(A)
    with pytest.raises(lib.SpcaError) as e:
        h.solve(1, 8, x0=G[:8], s=20.0, lowp_sweeps=3, engine=lib.SPCA_ENGINE_SIMT)
    assert e.value.status == lib.SPCA_E_UNSUPPORTED
    with pytest.raises(lib.SpcaError) as e:
        h.solve(1, 8, x0=G[:8], s=20.0, lowp_sweeps=-1)
    assert e.value.status == lib.SPCA_E_INVALID
    h.close()


def test_fp16_storage_handle(lib, spiked):
    A, G = spiked
    h32 = lib.Handle(A)
    h16 = lib.Handle(A, storage=lib.SPCA_FP16)
    a = h32.solve(2, 24, x0=G[:24], s=20.0, max_iter=30, tol=-1, lowp_sweeps=10)
    b = h16.solve(2, 24, x0=G[:24], s=20.0, max_iter=30, tol=-1, lowp_sweeps=10)
    h32.close()
    h16.close()
    assert a["objective"] == b["objective"]
    assert np.array_equal(a["support"], b["support"])


def _products_lowp(lib, h, form, X):
    import torch
    r, p = X.shape
    n = h.n
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    Ud = torch.zeros((r, n), dtype=torch.float32, device="cuda")
    Vd = torch.zeros((r, p), dtype=torch.float32, device="cuda")
    st = lib.spca_products(h.h, form, lib.SPCA_ENGINE_TC_LOWP, Xd.data_ptr(), p, r, Ud.data_ptr(), n, Vd.data_ptr(), p)
    assert st == 0, lib.spca_last_error(h.h)
    torch.cuda.synchronize()
    return Ud.cpu().numpy().astype(np.float64), Vd.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("storage,eps", [("fp16", 2.0 ** -12), ("fp8", 2.0 ** -4)])
@pytest.mark.parametrize("form", [1, 2])
def test_lowp_contractions_within_rounding(lib, spiked, storage, eps, form):
    """u = A x and v = A^T y on the low-precision copies.  Both operands are rounded to nearest
    with relative error at most eps (the leading FP16 plane: 2^-12; E4M3: 2^-4), each product then
    errs by at most (2 eps + eps^2) |a b|, and the FP32 sums add little: the error of every output
    stays below 2.1 eps of sum |a_k b_k| (E4M3 flushes entries below 2^-9 of the scaled range to
    zero, far below that).  y = +-1 (form 2) is exact in both formats."""
    A, G = spiked
    r = 40
    X = G[:r].copy()
    X[3, :: 2] = 0.0
    st = {"fp16": lib.SPCA_FP16, "fp8": lib.SPCA_FP8_E4M3_COLSCALED}[storage]
    h = lib.Handle(A, storage=st)
    U, V = _products_lowp(lib, h, form, X)
    h.close()
    A64, X64 = A.astype(np.float64), X.astype(np.float64)
    scale_u = np.abs(X64) @ np.abs(A64).T
    err_u = np.abs(U - X64 @ A64.T) / scale_u
    assert err_u.max() <= 2.1 * eps, err_u.max()
    Y = np.where(U >= 0, 1.0, -1.0) if form == 2 else U / np.linalg.norm(U, axis=1, keepdims=True)
    scale_v = np.abs(Y) @ np.abs(A64)
    err_v = np.abs(V - Y @ A64) / scale_v
    assert err_v.max() <= (1.1 if form == 2 else 2.1) * eps, err_v.max()
    # and the errors are rounding, not a misplaced operand: far below the bound on average
    assert np.median(err_u) <= 0.25 * eps and np.median(err_v) <= 0.25 * eps


def test_fp8_storage_handle(lib, spiked):
    A, G = spiked
    h8 = lib.Handle(A, storage=lib.SPCA_FP8_E4M3_COLSCALED)
    out = h8.solve(1, 24, x0=G[:24], s=20.0, max_iter=40, tol=-1, lowp_sweeps=10, want_starts=True)
    # FP32 sweeps (no low-precision ones) are those of an FP32 handle
    h32 = lib.Handle(A)
    a = h32.solve(1, 24, x0=G[:24], s=20.0, max_iter=30, tol=-1)
    b = h8.solve(1, 24, x0=G[:24], s=20.0, max_iter=30, tol=-1)
    h32.close()
    h8.close()
    assert a["objective"] == b["objective"] and np.array_equal(a["support"], b["support"])
    assert np.all(out["start_iters"] == 40)


def test_lowp_first_schedule(lib, oracle, spiked):
    """lowp_first = F runs F FP32 sweeps before the low-precision window (sweeps F+1 .. F+L), then
    FP32 again: a solve that stops at F sweeps is bit for bit the plain FP32 solve; no start
    stops inside the window or before two FP32 sweeps after it; every per-start objective is the
    FP64 objective of the returned x; and a window that starts after the basin is fixed leaves
    most starts where plain FP32 sweeps take them."""
    A, G = spiked
    r, F, L = 24, 6, 10
    h = lib.Handle(A)
    tc = lib.SPCA_ENGINE_TC   # the low-precision sweeps run on the tensor cores: compare like with like
    plain = h.solve(1, r, x0=G[:r], s=20.0, max_iter=F, tol=-1, engine=tc, want_starts=True)
    early = h.solve(1, r, x0=G[:r], s=20.0, max_iter=F, tol=-1, lowp_sweeps=L, lowp_first=F, engine=tc,
                    want_starts=True)
    assert np.array_equal(plain["start_x"], early["start_x"])
    out = h.solve(1, r, x0=G[:r], s=20.0, max_iter=60, tol=1e-6, lowp_sweeps=L, lowp_first=F, want_starts=True)
    ok = out["start_status"] != lib.SPCA_ST_DEGENERATE
    assert np.all(out["start_iters"][ok] >= F + L + 2)
    A64 = A.astype(np.float64)
    for c in range(r):
        fo, _ = oracle.objective(A64, 1, 0.0, out["start_x"][c].astype(np.float64))
        assert abs(out["start_objective"][c] - fo) <= 1e-9 * max(1.0, abs(fo))
    ref = h.solve(1, r, x0=G[:r], s=20.0, max_iter=60, tol=1e-6, engine=tc, want_starts=True)
    same = [np.array_equal(out["start_x"][c] != 0, ref["start_x"][c] != 0) for c in range(r)]
    assert np.mean(same) >= 0.75
    with pytest.raises(lib.SpcaError) as e:
        h.solve(1, r, x0=G[:r], s=20.0, lowp_sweeps=L, lowp_first=-1)
    assert e.value.status == lib.SPCA_E_INVALID
    h.close()
