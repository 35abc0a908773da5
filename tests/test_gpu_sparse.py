"""A sparse A in compressed sparse rows: the text corpora of Section 5 (document x word counts).

Step level: u = A x over the stored entries (a dense first-sweep x) and v = A^T y against FP64,
with rows long enough to be split into segments on both sides (a frequent word is in nearly every
document; the document-heavy case has documents of several thousand distinct words), and start
counts that leave ragged groups of 8 (and of 16: y = +-1 is packed in FP16).  Up to 32 starts
every output is an FP32 sum of at most 64 + 5 + (segments) rounded terms (a lane's FMA chain over
a strided subset of an item of at most 2048 entries, the warp's 5 reduction levels, the fix-up
over the row's segments), so its error is below (69 + segments) 2^-24 of sum |a_ij y_i|; for more
starts a lane sums a whole item (at most 2048 terms).

Solve level: every formulation against the FP64 oracle on the same starts (the oracle's own
products over the same stored entries); the sparse handle against a dense handle of the same
matrix; on-the-fly replacement; projection deflation (kept as a low-rank update of the sparse A)
against the FP64 deflated matrix, by products and by a sequence of components; edge cases (empty
rows and columns, no entries at all, repeated and unsorted input, device input) and the requests a
sparse handle refuses."""
import numpy as np
import pytest

from paper_1212_4137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sps = pytest.importorskip("scipy.sparse")


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1212_4137_gb300 import build, spca
    build.build()
    spca.load()
    return spca


def _bow(n, p, nnz, seed, **kw):
    ip, ix, v = I.bag_of_words(n, p, nnz, seed, **kw)
    return ip, ix, v, sps.csr_matrix((v.astype(np.float64), ix, ip), shape=(n, p))


def _products(lib, h, form, X):
    import torch
    r, p = X.shape
    n = h.n
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    Ud = torch.zeros((r, n + 3), dtype=torch.float32, device="cuda")
    Vd = torch.zeros((r, p + 1), dtype=torch.float32, device="cuda")
    st = lib.spca_products(h.h, form, lib.SPCA_ENGINE_AUTO, Xd.data_ptr(), p, r, Ud.data_ptr(), n + 3,
                           Vd.data_ptr(), p + 1)
    assert st == 0, lib.spca_last_error(h.h)
    torch.cuda.synchronize()
    return Ud[:, :n].cpu().numpy().astype(np.float64), Vd[:, :p].cpu().numpy().astype(np.float64)


def _bound(M64, r):
    """Up to 32 starts a lane sums a strided subset of an item (at most 2048 / 32 = 64 terms) and
    the warp adds the lanes' sums in 5 levels; more starts (slabs, lanes over starts) a lane sums
    a whole item (at most 2048 terms).  Split rows add their segments' sums in order."""
    longest = int(np.diff(M64.indptr).max())
    segs = -(-longest // 2048) if longest > 2048 else 0
    chain = 64 + 5 if r <= 32 else min(longest, 2048)
    return (chain + segs) * 2.0 ** -24


# (n, p, nnz, r): a word in nearly every document (long rows of A^T); documents of thousands of
# words (long rows of A); r = 1, a ragged last group, whole groups, several groups; more than 32
# starts (slabs of 64, lanes over starts), the last slab ragged
CASES = [(3000, 5000, 120000, 1), (3000, 5000, 120000, 13), (200, 20000, 600000, 8),
         (5000, 2000, 150000, 20), (700, 900, 9000, 64), (2000, 3000, 60000, 130)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("form", [1, 2])
def test_sparse_products_match_fp64(lib, case, form):
    n, p, nnz, r = case
    ip, ix, v, A64 = _bow(n, p, nnz, n + r)
    h = lib.Handle((ip, ix, v, (n, p)))
    rng = np.random.default_rng(n + p + r)
    X = rng.standard_normal((r, p)).astype(np.float32)
    if r > 2:
        X[1] = 0.0
        X[2, : p // 2] = 0.0
    U, V = _products(lib, h, form, X)
    h.close()
    X64 = X.astype(np.float64)
    AT64 = A64.T.tocsr()
    U_ref = (A64 @ X64.T).T
    scale_u = (abs(A64) @ np.abs(X64).T).T
    err_u = np.abs(U - U_ref) / (scale_u + 1e-30)
    assert err_u.max() <= _bound(A64, r), err_u.max()
    Yr = np.where(U >= 0, 1.0, -1.0) if form % 2 == 0 else U / np.maximum(np.linalg.norm(U, axis=1, keepdims=True),
                                                                           1e-300)
    V_ref = (AT64 @ Yr.T).T
    scale_v = (abs(AT64) @ np.abs(Yr).T).T
    live = np.linalg.norm(U, axis=1) > 0
    err_v = np.abs(V - V_ref)[live] / (scale_v[live] + 1e-30)
    assert err_v.max() <= _bound(AT64, r), err_v.max()


def _at_threshold(A64, form, x, gamma, s, rel=1e-4):
    """Entries whose selection one FP64 sweep from x decides within rel of its threshold: the s-th
    largest |v_i| (T_s) or gamma (U_gamma: v_i^2 against gamma)."""
    u = A64 @ x
    y = np.where(u >= 0, 1.0, -1.0) if form % 2 == 0 else u / np.linalg.norm(u)
    v = A64.T @ y
    if form in (5, 6):
        return np.abs(v * v - gamma) <= rel * gamma
    a = np.abs(v)
    t = np.sort(a)[::-1][s - 1]
    return np.abs(a - t) <= rel * t


@pytest.mark.parametrize("form", range(1, 9))
def test_sparse_solve_matches_oracle(lib, oracle, form):
    n, p, r = 800, 1500, 32
    ip, ix, v, A64 = _bow(n, p, 30000, 40 + form, topics=4, topic_words=8, topic_share=0.1)
    G = I.raw_starts(p, r, 41).astype(np.float32)
    kw = dict(s=5.0) if form <= 4 else dict(s=5.0, gamma_target=True, calib=6)
    h = lib.Handle((ip, ix, v, (n, p)))
    out = h.solve(form, r, x0=G, max_iter=100, tol=1e-9, want_starts=True, **kw)
    # iterates on fixed sweep counts (the FP32 stopping decision at tol 1e-9 is below FP32's
    # resolution of F, so converged runs stop a few sweeps apart)
    fixed = h.solve(form, r, x0=G, max_iter=25, tol=-1, want_starts=True, **kw)
    h.close()
    ref = oracle.solve(A64, form, G.astype(np.float64), max_iter=100, tol=1e-9, **kw)
    key_gpu = out["explained_variance"] if form >= 5 else out["objective"]
    key_ref = ref.ev[ref.best] if form >= 5 else ref.f[ref.best]
    assert abs(key_gpu - key_ref) <= 1e-5 * abs(key_ref), (key_gpu, key_ref)
    assert np.mean(out["start_status"] == ref.status) >= 0.9
    # the objective of every returned x is its FP64 value
    for c in range(0, r, 7):
        fo, _ = oracle.objective(A64, form, out["start_gamma"][c], out["start_x"][c].astype(np.float64))
        assert abs(out["start_objective"][c] - fo) <= 1e-9 * max(1.0, abs(fo)), c
    ref = oracle.solve(A64, form, G.astype(np.float64), max_iter=25, tol=-1, **kw)
    X, out = fixed["start_x"], fixed
    same = [c for c in range(r) if np.array_equal(X[c] != 0, ref.X[c] != 0)]
    for c in same:
        assert np.max(np.abs(X[c] - ref.X[c])) <= 1e-4, c
    # A start on another support differs from the oracle's only in entries at the selection
    # threshold, or in entries near zero (the continuous operators of forms 3, 4, 7 and 8).  For
    # forms 5 and 6 the Section 4.1 rule freezes gamma at the (s+1)-th largest v_i^2, so from then
    # on one entry sits at the threshold in every start and rounding decides it in any sweep; a
    # start that took it in at another sweep than the oracle follows another path, and only the
    # share of matching starts bounds those (as for the dense fixed-sweep runs).
    if form not in (5, 6):
        for c in set(range(r)) - set(same):
            moved = (X[c] != 0) != (ref.X[c] != 0)
            assert np.all(_at_threshold(A64, form, X[c].astype(np.float64), out["start_gamma"][c], 5)[moved]
                          | (np.maximum(np.abs(X[c]), np.abs(ref.X[c])) <= 1e-3)[moved]), c
    assert len(same) >= r // 2


@pytest.mark.parametrize("form", [1, 4, 6])
def test_sparse_handle_matches_dense_handle(lib, form):
    n, p, r = 600, 1000, 24
    ip, ix, v, A64 = _bow(n, p, 20000, 50 + form)
    G = I.raw_starts(p, r, 51).astype(np.float32)
    kw = dict(s=5.0) if form <= 4 else dict(s=5.0, gamma_target=True, calib=6)
    hs = lib.Handle((ip, ix, v, (n, p)))
    hd = lib.Handle(A64.toarray().astype(np.float32))
    a = hs.solve(form, r, x0=G, max_iter=60, tol=1e-9, want_starts=True, **kw)
    b = hd.solve(form, r, x0=G, max_iter=60, tol=1e-9, want_starts=True, engine=lib.SPCA_ENGINE_SIMT, **kw)
    hs.close()
    hd.close()
    fa, fb = a["start_objective"], b["start_objective"]
    same = np.array([np.array_equal(a["start_x"][c] != 0, b["start_x"][c] != 0) for c in range(r)])
    assert np.max(np.abs(fa[same] - fb[same]) / np.abs(fb[same])) <= 1e-6
    # other supports differ in entries at the selection threshold only (with gamma frozen by the
    # Section 4.1 rule at a converged start, an entry sits at it), which moves f by ~0
    for c in np.flatnonzero(~same):
        moved = (a["start_x"][c] != 0) != (b["start_x"][c] != 0)
        assert np.all(_at_threshold(A64, form, b["start_x"][c].astype(np.float64), b["start_gamma"][c], 5)[moved]), c
        assert abs(fa[c] - fb[c]) <= 1e-5 * abs(fb[c]), c
    assert abs(a["objective"] - b["objective"]) <= 1e-5 * abs(b["objective"])


def test_sparse_otf_matches_plain(lib):
    n, p, l, r = 700, 1200, 40, 8
    ip, ix, v, _ = _bow(n, p, 15000, 60)
    G = I.raw_starts(p, l, 61).astype(np.float32)
    h = lib.Handle((ip, ix, v, (n, p)))
    kw = dict(s=5.0, max_iter=30, tol=-1, want_starts=True)
    plain = h.solve(1, l, x0=G, **kw)
    otf = h.solve(1, r, x0=G, total_starts=l, **kw)
    h.close()
    assert otf["sweeps_total"] == 30 * l
    fp, fo = plain["start_objective"], otf["start_objective"]
    assert np.max(np.abs(fo - fp) / np.abs(fp)) <= 1e-6
    assert abs(otf["objective"] - plain["objective"]) <= 1e-6 * plain["objective"]


def test_sparse_edge_cases(lib, oracle):
    import torch
    n, p = 300, 400
    ip, ix, v, A64 = _bow(n, p, 3000, 70)
    # empty rows and columns: drop every entry of rows 0..49 and of columns 0..99
    M = A64.tolil()
    M[:50, :] = 0
    M[:, :100] = 0
    M = M.tocsr()
    M.eliminate_zeros()
    G = I.raw_starts(p, 6, 71).astype(np.float32)
    h = lib.Handle((M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float32), (n, p)))
    out = h.solve(3, 6, s=4.0, x0=G, max_iter=50, tol=1e-9)
    h.close()
    ref = oracle.solve(M, 3, G.astype(np.float64), s=4.0, max_iter=50, tol=1e-9)
    assert abs(out["objective"] - ref.f[ref.best]) <= 1e-5 * ref.f[ref.best]
    # no entries at all: every start ends degenerate with x = 0
    h = lib.Handle((np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32), (n, p)))
    for form in (1, 2, 7):
        out = h.solve(form, 4, s=3.0, gamma=0.1, max_iter=10, tol=1e-9, want_starts=True)
        assert np.all(out["start_status"] == lib.SPCA_ST_DEGENERATE) and out["objective"] == 0.0
    h.close()
    # repeated and unsorted entries: the same handle as the canonical matrix, bit for bit
    rng = np.random.default_rng(72)
    rows = np.repeat(np.arange(n), np.diff(ip))
    perm = np.lexsort((rng.uniform(size=ix.size), rows))        # shuffle columns within rows
    half = v[perm] / 2
    ip2 = ip * 2
    ix2 = np.repeat(ix[perm], 2)
    v2 = np.repeat(half, 2).astype(np.float32)                   # each entry as two halves
    G = I.raw_starts(p, 5, 73).astype(np.float32)
    outs = []
    for arrays in ((ip, ix, v), (ip2, ix2, v2)):
        h = lib.Handle((*arrays, (n, p)))
        outs.append(h.solve(2, 5, s=4.0, x0=G, max_iter=30, tol=1e-9, want_starts=True))
        h.close()
    assert np.array_equal(outs[0]["start_x"], outs[1]["start_x"])
    # device input
    d = [torch.from_numpy(a).cuda() for a in (ip, ix, v)]
    st, hh = lib.spca_create_csr(n, p, int(ip[-1]), d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), True)
    assert st == 0
    hdev = lib.Handle.__new__(lib.Handle)
    hdev.h, hdev.n, hdev.p = hh, n, p
    o = hdev.solve(2, 5, s=4.0, x0=G, max_iter=30, tol=1e-9, want_starts=True)
    assert np.array_equal(o["start_x"], outs[0]["start_x"])
    # what a sparse handle refuses
    with pytest.raises(lib.SpcaError) as e:
        hdev.solve(1, 4, s=3.0, engine=lib.SPCA_ENGINE_TC)
    assert e.value.status == lib.SPCA_E_UNSUPPORTED
    with pytest.raises(lib.SpcaError) as e:
        hdev.solve(1, 4, s=3.0, lowp_sweeps=2)
    assert e.value.status == lib.SPCA_E_UNSUPPORTED
    hdev.close()


def test_sparse_invalid_input(lib):
    n, p = 5, 6
    good = (np.array([0, 1, 2, 2, 3, 4], np.int64), np.array([0, 5, 2, 3], np.int32), np.ones(4, np.float32))
    st, h = lib.spca_create_csr(n, p, 4, *good, False)
    assert st == 0
    lib.spca_destroy(h)
    bad = [
        (np.array([0, 1, 2, 2, 3, 5], np.int64), good[1], good[2]),      # row_ptr[n] != nnz
        (np.array([0, 2, 1, 2, 3, 4], np.int64), good[1], good[2]),      # decreasing
        (good[0], np.array([0, 6, 2, 3], np.int32), good[2]),            # column out of range
        (good[0], np.array([0, -1, 2, 3], np.int32), good[2]),
        (good[0], good[1], np.array([1, np.nan, 1, 1], np.float32)),     # not finite
    ]
    for ip, ix, v in bad:
        st, h = lib.spca_create_csr(n, p, 4, ip, ix, v, False)
        assert st == lib.SPCA_E_INVALID and not h
    st, h = lib.spca_create_csr(0, p, 0, np.zeros(1, np.int64), good[1], good[2], False)
    assert st == lib.SPCA_E_INVALID


@pytest.mark.parametrize("r", [24, 48])
@pytest.mark.parametrize("form", [1, 2])
def test_sparse_deflated_products_match_fp64(lib, oracle, form, r):
    """A_2 = A (I - z1 z1^T)(I - z2 z2^T) = A - W Z^T, w_i = A_{i-1} z_i: the GPU keeps A sparse and
    subtracts W (Z^T x) and Z (W^T y).  Its errors are relative to the sizes of both parts."""
    n, p = 700, 1900
    ip, ix, v, A64 = _bow(n, p, 30000, 80 + r)
    rng = np.random.default_rng(81)
    xs = [rng.standard_normal(p).astype(np.float32) * 3.0 for _ in range(2)]
    D = A64.toarray()
    zs, ws = [], []
    for x in xs:
        z = x.astype(np.float64) / np.linalg.norm(x.astype(np.float64))
        ws.append(D @ z)
        zs.append(z)
        D = oracle.deflate(D, x.astype(np.float64))
    h = lib.Handle((ip, ix, v, (n, p)))
    for x in xs:
        h.deflate(x)
    X = rng.standard_normal((r, p)).astype(np.float32)
    X[1] = xs[1]                                                   # A_2 z2 = 0
    U, V = _products(lib, h, form, X)
    h.close()
    X64 = X.astype(np.float64)
    absA = abs(A64)
    scale_u = (absA @ np.abs(X64).T).T + sum(np.outer(np.abs(X64 @ z), np.abs(w)) for z, w in zip(zs, ws))
    assert np.max(np.abs(U - X64 @ D.T) / (scale_u + 1e-300)) <= 2e-5
    Y = np.where(U >= 0, 1.0, -1.0) if form == 2 else U / np.linalg.norm(U, axis=1, keepdims=True)
    scale_v = (absA.T @ np.abs(Y).T).T + sum(np.outer(np.abs(Y @ w), np.abs(z)) for z, w in zip(zs, ws))
    live = np.linalg.norm(U, axis=1) > 0
    assert np.max((np.abs(V - Y @ D) / (scale_v + 1e-300))[live]) <= 2e-5


def test_sparse_components_match_fp64_sequence(lib, oracle):
    """Several components of a bag of words (formulation 1, s = 5, as for the text corpora): each
    solve, then deflation by its x; the objective and support of every component match the FP64
    sequence (oracle solve on the densified deflated matrix, oracle deflation by the oracle's x)."""
    n, p, r = 600, 900, 24
    ip, ix, v, A64 = _bow(n, p, 20000, 90, topics=4, topic_words=6, topic_share=0.15)
    G = I.raw_starts(p, r, 91).astype(np.float32)
    h = lib.Handle((ip, ix, v, (n, p)))
    D64 = A64.toarray()
    for comp in range(4):
        out = h.solve(1, r, s=5.0, x0=G, max_iter=200, tol=1e-9)
        ref = oracle.solve(D64, 1, G.astype(np.float64), s=5.0, max_iter=200, tol=1e-9)
        xr = ref.X[ref.best]
        assert abs(out["objective"] - ref.f[ref.best]) <= 1e-5 * ref.f[ref.best], (comp, out["objective"])
        assert np.array_equal(out["support"], np.flatnonzero(xr)), comp
        h.deflate(out["x"])
        D64 = oracle.deflate(D64, xr)
    h.close()
