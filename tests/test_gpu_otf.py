"""On-the-fly replacement (Section 4.3): l starts run through r < l slots, a slot taking the next
start in the sweep its start stops.  A start's iterates do not depend on the other starts, so every
start must end as it does in a plain solve of all l starts at once (up to the contraction's
rounding, which depends on how many starts share a tile), and the best start must match the FP64
oracle's over the l starts."""
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
    n, p = 300, 900
    return I.spiked_matrix(n, p, I.spiked_thetas(n, p), 15, 71, dtype=np.float32)


@pytest.mark.parametrize("source", ["seeded", "host", "device"])
def test_otf_starts_end_as_in_a_plain_solve(lib, spiked, source):
    import torch
    A = spiked
    l, r, p = 48, 12, A.shape[1]
    G = I.raw_starts(p, l, 72).astype(np.float32)
    h = lib.Handle(A)
    kw = dict(s=10.0, max_iter=20, tol=-1, want_starts=True, seed=73)
    if source == "seeded":
        plain = h.solve(1, l, **kw)
        otf = h.solve(1, r, total_starts=l, **kw)
    elif source == "host":
        plain = h.solve(1, l, x0=G, **kw)
        otf = h.solve(1, r, x0=G, total_starts=l, **kw)
    else:
        Gd = torch.from_numpy(G).cuda()
        plain = h.solve(1, l, x0=Gd.data_ptr(), x0_device=True, **kw)
        otf = h.solve(1, r, x0=Gd.data_ptr(), x0_device=True, total_starts=l, **kw)
    h.close()
    assert np.all(otf["start_iters"] == 20) and np.all(otf["start_status"] == lib.SPCA_ST_MAXITER)
    assert otf["sweeps_total"] == 20 * l
    fp, fo = plain["start_objective"], otf["start_objective"]
    assert np.max(np.abs(fo - fp) / np.abs(fp)) <= 1e-6
    same = [c for c in range(l) if np.array_equal(otf["start_x"][c] != 0, plain["start_x"][c] != 0)]
    assert len(same) >= int(0.95 * l)
    for c in same:
        assert np.max(np.abs(otf["start_x"][c] - plain["start_x"][c])) <= 1e-4
    assert abs(otf["objective"] - plain["objective"]) <= 1e-6 * plain["objective"]


@pytest.mark.parametrize("form", [1, 5, 8])
def test_otf_best_matches_oracle(lib, oracle, spiked, form):
    A = spiked
    l, r, p = 40, 8, A.shape[1]
    G = I.raw_starts(p, l, 74).astype(np.float32)
    kw = dict(s=10.0) if form <= 4 else dict(s=10.0, gamma_target=True, calib=6)
    h = lib.Handle(A)
    out = h.solve(form, r, x0=G, total_starts=l, max_iter=100, tol=1e-9, want_starts=True, **kw)
    h.close()
    ref = oracle.solve(A.astype(np.float64), form, G.astype(np.float64), max_iter=100, tol=1e-9, **kw)
    key_gpu = out["explained_variance"] if form >= 5 else out["objective"]
    key_ref = ref.ev[ref.best] if form >= 5 else ref.f[ref.best]
    assert abs(key_gpu - key_ref) <= 1e-5 * abs(key_ref), (key_gpu, key_ref)
    assert out["sweeps_total"] == int(out["start_iters"].sum())
    assert np.all(out["start_iters"] >= 1)
    # the starts' statuses agree with the oracle's on nearly every start
    assert np.mean(out["start_status"] == ref.status) >= 0.9


def test_otf_rejects_low_precision_sweeps(lib, spiked):
    h = lib.Handle(spiked)
    with pytest.raises(lib.SpcaError) as e:
        h.solve(1, 8, s=10.0, total_starts=32, lowp_sweeps=3)
    assert e.value.status == lib.SPCA_E_UNSUPPORTED
    h.close()
