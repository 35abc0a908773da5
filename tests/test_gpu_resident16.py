"""Resident 16-bit handles (storage SPCA_FP16_RESIDENT): A kept on the device only as the leading
FP16 planes of A and of A^T with their power-of-two row scales, 4 bytes per entry instead of 16.
Every sweep is a low-precision sweep, and the matrix the finalise evaluates is the 16-bit copy of
A^T: column j of A times 2^e_j (e_j = 13 - floor(log2 max_i |a_ij|)), rounded to FP16 to nearest,
times 2^-e_j.  That copy is rebuilt here on the host, independently of the library, from that
definition.

Checked: every reported per-start objective is the FP64 objective (Table 1) of the returned x on
the 16-bit copy; the handle really holds 4 bytes per entry; the best objective stays within the
precision bar (1e-3 relative) of a plain FP32 solve; the low-precision products equal those of an
SPCA_FP16 handle bit for bit (the same leading planes); a resident member of a group gives the
same bits alone and in a mix, and agrees with its solo solve; refusals."""
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
    A = I.spiked_matrix(n, p, I.spiked_thetas(n, p), 20, 911, dtype=np.float32)
    G = I.raw_starts(p, 64, 912).astype(np.float32)
    return A, G


def copy16(A):
    """The 16-bit copy of A as its transpose's rows hold it: per column j of A the scale 2^e_j with
    e_j = 13 - floor(log2 max |A[:, j]|) (0 for a zero column, clamped to [-120, 120]), FP16
    round-to-nearest-even of the scaled column, unscaled in FP64."""
    A = np.asarray(A, np.float32)
    m = np.abs(A).max(axis=0).astype(np.float64)
    e = np.zeros(A.shape[1], np.int64)
    nz = m > 0
    e[nz] = np.clip(13 - (np.frexp(m[nz])[1] - 1), -120, 120)
    scale = np.ldexp(np.float32(1.0), e).astype(np.float32)
    hi = (A * scale[None, :]).astype(np.float16)
    return hi.astype(np.float64) / scale.astype(np.float64)[None, :]


def _kw(form):
    return dict(s=20.0) if form <= 4 else dict(s=20.0, gamma_target=True, calib=8)


def test_copy16_definition():
    """The host copy itself: exact FP16 values of the scaled columns, within half an FP16 ulp."""
    rng = np.random.default_rng(3)
    A = (rng.standard_normal((50, 40)) * np.exp(rng.uniform(-20, 20, 40))[None, :]).astype(np.float32)
    A[:, 5] = 0.0
    C = copy16(A)
    assert np.all(C[:, 5] == 0.0)
    nz = np.abs(A).max(axis=0) > 0
    rel = np.abs(C - A)[:, nz] / np.abs(A).max(axis=0)[nz][None, :]
    assert rel.max() <= 2.0 ** -11 * 1.0001   # half an FP16 ulp (4) against a scaled maximum >= 2^13
    assert rel.max() >= 2.0 ** -16            # and it is a rounding, not a copy
    # the largest entry of each nonzero column lands in [2^13, 2^14) after scaling
    m = np.abs(A).max(axis=0)
    e = 13 - (np.frexp(m[m > 0])[1] - 1)
    assert np.all((np.ldexp(m[m > 0], e) >= 2 ** 13) & (np.ldexp(m[m > 0], e) < 2 ** 14))


@pytest.mark.parametrize("form", range(1, 9))
def test_resident_objective_is_that_of_the_copy(lib, oracle, spiked, form):
    A, G = spiked
    C = copy16(A)
    h = lib.Handle(A, storage=lib.SPCA_FP16_RESIDENT)
    r = 24
    out = h.solve(form, r, x0=G[:r], max_iter=60, tol=1e-7, want_starts=True, **_kw(form))
    h.close()
    assert out["sweeps_total"] > 0
    for c in range(r):
        fo, evo = oracle.objective(C, form, out["start_gamma"][c], out["start_x"][c].astype(np.float64))
        assert abs(out["start_objective"][c] - fo) <= 1e-9 * max(1.0, abs(fo)), (c, out["start_objective"][c], fo)
        assert abs(out["start_explained"][c] - evo) <= 1e-9 * max(1.0, abs(evo))
    b = out["best_start"]
    assert np.array_equal(out["support"], np.flatnonzero(out["start_x"][b]))


def test_resident_holds_four_bytes_per_entry(lib):
    import torch
    n, p = 4000, 20000
    A = I.gaussian_matrix(n, p, 5).astype(np.float32)
    Ad = torch.from_numpy(A).cuda()
    torch.cuda.synchronize()

    def drop(storage):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        h = lib.Handle(Ad, storage=storage)
        torch.cuda.synchronize()
        used = free0 - torch.cuda.mem_get_info()[0]
        h.close()
        return used

    full, res = drop(lib.SPCA_F32), drop(lib.SPCA_FP16_RESIDENT)
    entries = n * p
    assert full >= 15 * entries               # FP32 A and A^T, two FP16 planes of each
    assert res <= 4 * entries + (64 << 20)    # the two leading planes, scales, stream-K scratch


@pytest.mark.parametrize("form", [1, 2])
def test_resident_within_precision_bar(lib, spiked, form):
    A, G = spiked
    r = 64
    h32 = lib.Handle(A)
    ref = h32.solve(form, r, x0=G, s=20.0, max_iter=100, tol=1e-9)
    h32.close()
    h = lib.Handle(A, storage=lib.SPCA_FP16_RESIDENT)
    out = h.solve(form, r, x0=G, s=20.0, max_iter=100, tol=1e-9)
    h.close()
    assert abs(out["objective"] - ref["objective"]) <= 1e-3 * abs(ref["objective"])


def test_resident_products_are_the_fp16_handles_leading_planes(lib, spiked):
    import torch
    A, G = spiked
    r = 40
    n, p = A.shape
    X = torch.from_numpy(np.ascontiguousarray(G[:r])).cuda()
    outs = []
    for storage in (lib.SPCA_FP16, lib.SPCA_FP16_RESIDENT):
        h = lib.Handle(A, storage=storage)
        U = torch.zeros((r, n), dtype=torch.float32, device="cuda")
        V = torch.zeros((r, p), dtype=torch.float32, device="cuda")
        st = lib.spca_products(h.h, 1, lib.SPCA_ENGINE_TC_LOWP, X.data_ptr(), p, r, U.data_ptr(), n, V.data_ptr(), p)
        assert st == 0, lib.spca_last_error(h.h)
        torch.cuda.synchronize()
        outs.append((U.cpu().numpy(), V.cpu().numpy()))
        h.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_resident_in_groups(lib, spiked):
    A, G = spiked
    B = I.spiked_matrix(500, 1800, I.spiked_thetas(500, 1800), 15, 913, dtype=np.float32)
    GB = I.raw_starts(1800, 32, 914).astype(np.float32)
    ha = lib.Handle(A, storage=lib.SPCA_FP16_RESIDENT)
    hb = lib.Handle(B)
    hc = lib.Handle(B, storage=lib.SPCA_FP16_RESIDENT)
    pa = (ha, 2, 48, dict(x0=G[:48], s=20.0, max_iter=40, tol=-1))
    pb = (hb, 5, 32, dict(x0=GB, s=15.0, gamma_target=True, calib=6, max_iter=40, tol=-1))
    pc = (hc, 1, 32, dict(x0=GB, s=15.0, max_iter=40, tol=-1))
    # a wide resident pool on another matrix: the group's tiles become 256 columns wide
    D = I.spiked_matrix(400, 1500, I.spiked_thetas(400, 1500), 15, 915, dtype=np.float32)
    hd = lib.Handle(D, storage=lib.SPCA_FP16_RESIDENT)
    pd = (hd, 1, 300, dict(seed=5, s=15.0, max_iter=40, tol=-1))
    g = lib.Group()
    alone = g.solve([pa], want_starts=True)[0]
    mix = g.solve([pb, pa, pc], want_starts=True)      # resident and FP32 members together
    wide = g.solve([pa, pd], want_starts=True)         # resident members only, 256-wide tiles
    g.close()
    hd.close()
    for other in (mix[1], wide[0]):
        assert np.array_equal(alone["start_x"], other["start_x"])
        assert alone["objective"] == other["objective"]
    # against solo solves on the same handles (another contraction kernel: rounding order differs)
    for (hh, form, r, kw), o in zip((pb, pa, pc), mix):
        solo = hh.solve(form, r, want_starts=True, **kw)
        close = np.abs(o["start_objective"] - solo["start_objective"]) <= 1e-4 * np.maximum(
            1.0, np.abs(solo["start_objective"]))
        assert np.mean(close) >= 0.9, (form, np.mean(close))
        assert abs(o["objective"] - solo["objective"]) <= 1e-4 * abs(solo["objective"])
    for hh in (ha, hb, hc):
        hh.close()


def test_resident_refusals(lib, spiked):
    import torch
    A, G = spiked
    h = lib.Handle(A, storage=lib.SPCA_FP16_RESIDENT)
    for kw, code in ((dict(engine=lib.SPCA_ENGINE_SIMT), lib.SPCA_E_UNSUPPORTED),
                     (dict(lowp_sweeps=5), lib.SPCA_E_INVALID),
                     (dict(refine_sweeps=5), lib.SPCA_E_INVALID),
                     (dict(total_starts=64), lib.SPCA_E_UNSUPPORTED)):
        with pytest.raises(lib.SpcaError) as e:
            h.solve(1, 16, seed=1, s=20.0, **kw)
        assert e.value.status == code, kw
    x = np.zeros(A.shape[1], np.float32)
    x[:5] = 1.0
    assert lib.spca_deflate(h.h, x) == lib.SPCA_E_UNSUPPORTED
    X = torch.from_numpy(np.ascontiguousarray(G[:8])).cuda()
    U = torch.zeros((8, A.shape[0]), dtype=torch.float32, device="cuda")
    V = torch.zeros((8, A.shape[1]), dtype=torch.float32, device="cuda")
    assert lib.spca_products(h.h, 1, lib.SPCA_ENGINE_TC, X.data_ptr(), A.shape[1], 8, U.data_ptr(), A.shape[0],
                             V.data_ptr(), A.shape[1]) == lib.SPCA_E_UNSUPPORTED
    # still usable
    out = h.solve(1, 16, x0=G[:16], s=20.0, max_iter=10, tol=-1)
    assert out["sweeps_total"] == 160
    h.close()
