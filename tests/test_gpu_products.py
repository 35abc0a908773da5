"""Step-level parity of the two contractions of a sweep (u = A x, y-step, v = A^T y) for both
engines (FP32 CUDA cores; tcgen05 tensor cores on two row-scaled FP16 planes per FP32 operand)
against FP64, on shapes that span several tiles and ragged tails.  The tensor-core engine keeps
22 significant bits of every operand and sums every plane product above the 2^-21 relative
level, so both engines must agree with FP64 to FP32 accumulation accuracy."""
import numpy as np
import pytest

from paper_1212_4137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# the CTA-pair contraction splits tiles over its resident pairs along K (stream-K): the shapes
# include tiles cut into 16 one-K-block parts (300 x 1003 x 40) and a single start with a long
# K (4000 x 300 x 1: each tile in about 38 parts), as well as whole tiles
# and few starts with rows longer than the streaming GEMV's shared memory holds (1200 x 17000 x 5:
# u = A x streams x in three chunks of 6400 columns)
SHAPES = [(7, 9, 3), (300, 1003, 40), (129, 257, 300), (1000, 3000, 257), (2500, 700, 520), (4000, 300, 1),
          (1200, 17000, 5)]


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1212_4137_gb300 import build, spca
    build.build()
    spca.load()
    return spca


def _bound(engine, K):
    """Error bound relative to sum_k |a_k b_k|.  FP32 FMA chains (CUDA cores) round to nearest:
    2e-6 covers K up to a few thousand.  The tensor core's FP32 accumulator truncates once per
    MMA step (K/16 steps for the hi x hi accumulator), losing less than one ulp (2^-23
    relative) each time, and on a sum whose terms share one sign these losses add up."""
    if engine == "simt":
        return 2e-6
    return max(2e-6, (K / 16.0) * 2.0 ** -23)


def _run(lib, h, form, engine, X):
    import torch
    r, p = X.shape
    n = h.n
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    Ud = torch.zeros((r, n + 1), dtype=torch.float32, device="cuda")
    Vd = torch.zeros((r, p + 5), dtype=torch.float32, device="cuda")
    st = lib.spca_products(h.h, form, engine, Xd.data_ptr(), p, r, Ud.data_ptr(), n + 1, Vd.data_ptr(), p + 5)
    assert st == 0, lib.spca_last_error(h.h)
    torch.cuda.synchronize()
    return Ud[:, :n].cpu().numpy().astype(np.float64), Vd[:, :p].cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("engine", ["simt", "tc"])
@pytest.mark.parametrize("form", [1, 2])
def test_products_match_fp64(lib, shape, engine, form):
    n, p, r = shape
    A = I.gaussian_matrix(n, p, 500 + n).astype(np.float32)
    A64 = A.astype(np.float64)
    rng = np.random.default_rng(n + p)
    X = rng.standard_normal((r, p)).astype(np.float32)
    X[:, rng.uniform(size=p) < 0.5] = 0.0            # sparse-ish iterates as after an x-step
    X[0] = 0.0
    X[0, p // 2] = 1.0
    eng = {"simt": lib.SPCA_ENGINE_SIMT, "tc": lib.SPCA_ENGINE_TC}[engine]
    h = lib.Handle(A)
    U, V = _run(lib, h, form, eng, X)
    h.close()
    U_ref = X.astype(np.float64) @ A64.T                      # r x n
    scale_u = np.abs(X.astype(np.float64)) @ np.abs(A64).T    # bound of the rounding error
    err_u = np.abs(U - U_ref) / (scale_u + 1e-30)
    assert err_u.max() <= _bound(engine, p), err_u.max()
    # y from the GPU's own u (same sign / scale decisions), then v in FP64
    if form % 2 == 0:
        Yr = np.where(U >= 0, 1.0, -1.0)
    else:
        Yr = U / np.linalg.norm(U, axis=1, keepdims=True)
    V_ref = Yr @ A64
    scale_v = np.abs(Yr) @ np.abs(A64)
    err = np.abs(V - V_ref) / (scale_v + 1e-30)
    assert err.max() <= _bound(engine, n), err.max()


def test_engines_agree_on_spiked(lib):
    n, p, r = 600, 2100, 130
    A = I.spiked_matrix(n, p, I.spiked_thetas(n, p), 20, 501, dtype=np.float32)
    G = I.raw_starts(p, r, 502).astype(np.float32)
    h = lib.Handle(A)
    for form in (1, 2):
        Us, Vs = _run(lib, h, form, lib.SPCA_ENGINE_SIMT, G)
        Ut, Vt = _run(lib, h, form, lib.SPCA_ENGINE_TC, G)
        assert np.abs(Us - Ut).max() <= 1e-5 * np.abs(Us).max()
        assert np.abs(Vs - Vt).max() <= 1e-5 * np.abs(Vs).max()
    h.close()


@pytest.mark.parametrize("form", [1, 2])
def test_products_with_column_scales(lib, form):
    """Columns of A spread over twelve orders of magnitude: the tensor-core operands carry one
    power-of-two scale per row of A (u = A x) and per row of A^T (v = A^T y), so every entry of
    v = A^T y keeps its relative accuracy whatever its column's magnitude, and u = A x keeps the
    bound relative to sum |a_k x_k|."""
    n, p, r = 900, 1500, 70
    rng = np.random.default_rng(77)
    A = (I.gaussian_matrix(n, p, 78) * 10.0 ** rng.uniform(-6, 6, size=p)).astype(np.float32)
    A64 = A.astype(np.float64)
    X = rng.standard_normal((r, p)).astype(np.float32)
    X[:, rng.uniform(size=p) < 0.5] = 0.0
    h = lib.Handle(A)
    U, V = _run(lib, h, form, lib.SPCA_ENGINE_TC, X)
    h.close()
    err_u = np.abs(U - X.astype(np.float64) @ A64.T) / (np.abs(X.astype(np.float64)) @ np.abs(A64).T + 1e-300)
    assert err_u.max() <= _bound("tc", p), err_u.max()
    Yr = np.where(U >= 0, 1.0, -1.0) if form % 2 == 0 else U / np.linalg.norm(U, axis=1, keepdims=True)
    err_v = np.abs(V - Yr @ A64) / (np.abs(Yr) @ np.abs(A64) + 1e-300)
    assert err_v.max() <= _bound("tc", n), err_v.max()
