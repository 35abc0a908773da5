"""spca_objective_noalloc: the per-start objective and explained variance for callers that
cannot allocate device memory (inside a foreign graph capture, under an allocator that owns the
device, in a latency-critical loop).  Its values must equal what spca_solve reports for the same
x's (start_objective, start_explained), within the objective tolerance of the parity tests, on
two calls in a row that share the scratch array.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1212_4137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

OBJ_RTOL = 1e-5


def _check(ref, got):
    ref = np.asarray(ref, np.float64)
    assert np.all(np.abs(got - ref) <= OBJ_RTOL * np.maximum(1.0, np.abs(ref))), np.max(np.abs(got - ref))


def test_objective_noalloc_matches_solve():
    import torch
    assert torch.cuda.is_available()
    from paper_1212_4137_gb300 import build, spca
    build.build()
    spca.load()
    n, p = 300, 1003
    A = I.spiked_matrix(n, p, I.spiked_thetas(n, p), 12, 11, dtype=np.float32)
    Ad = torch.from_numpy(A).cuda()
    h = spca.Handle(A)
    cases = [(1, 40, dict(s=12)), (8, 25, dict(gamma=2.0)), (4, 40, dict(s=12.0))]
    for call, (form, r, kw) in enumerate(cases):
        G = I.raw_starts(p, r, 600 + call).astype(np.float32)
        out = h.solve(form, r, max_iter=20, tol=-1, x0=G, want_starts=True, **kw)
        X = torch.from_numpy(out["start_x"]).cuda()
        f = torch.full((r,), np.nan, dtype=torch.float64, device="cuda")
        ev = torch.full((r,), np.nan, dtype=torch.float64, device="cuda")
        st = spca.spca_objective_noalloc(form, kw.get("gamma", 0.0), Ad.data_ptr(), n, p, p, X.data_ptr(), p, r,
                                         f.data_ptr(), ev.data_ptr(), 0)
        assert st == spca.SPCA_OK
        torch.cuda.synchronize()
        _check(out["start_objective"], f.cpu().numpy())
        _check(out["start_explained"], ev.cpu().numpy())
    h.close()
    # sizes beyond the fixed scratch are refused before anything runs
    r_big = 262144 // ((n + 255) // 256) + 1
    st = spca.spca_objective_noalloc(1, 0.0, Ad.data_ptr(), n, p, p, Ad.data_ptr(), p, r_big, Ad.data_ptr(),
                                     Ad.data_ptr(), 0)
    assert st == spca.SPCA_E_INVALID
