"""spca_objective_noalloc: the per-start objective and explained variance for callers that
cannot allocate device memory (inside a foreign graph capture, under an allocator that owns the
device, in a latency-critical loop).  Its values must equal the FP64 oracle's objective of the
same x's, for all eight formulations, and what spca_solve reports for them (start_objective,
start_explained), within the objective tolerance of the parity tests, on calls in a row that
share the one scratch array.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1212_4137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

OBJ_RTOL = 1e-5
GAMMA = {5: 0.5, 6: 60.0, 7: 0.2, 8: 2.0}


def _close(ref, got):
    ref = np.asarray(ref, np.float64)
    err = np.abs(got - ref)
    assert np.all(err <= OBJ_RTOL * np.maximum(1.0, np.abs(ref))), np.max(err)


def test_objective_noalloc_matches_oracle_and_solve(oracle):
    import torch
    assert torch.cuda.is_available()
    from paper_1212_4137_gb300 import build, spca
    build.build()
    spca.load()
    n, p = 300, 1003
    A = I.spiked_matrix(n, p, I.spiked_thetas(n, p), 12, 11, dtype=np.float32)
    A64 = A.astype(np.float64)
    Ad = torch.from_numpy(A).cuda()
    h = spca.Handle(A)
    for form in range(1, 9):
        r = 24 + 3 * form
        kw = dict(s=12) if form <= 4 else dict(gamma=GAMMA[form])
        G = I.raw_starts(p, r, 600 + form).astype(np.float32)
        out = h.solve(form, r, max_iter=20, tol=-1, x0=G, want_starts=True, **kw)
        X = torch.from_numpy(out["start_x"]).cuda()
        gamma = kw.get("gamma", 0.0)
        # two calls in a row on the shared scratch: both must give the same values
        for call in range(2):
            f = torch.full((r,), np.nan, dtype=torch.float64, device="cuda")
            ev = torch.full((r,), np.nan, dtype=torch.float64, device="cuda")
            st = spca.spca_objective_noalloc(form, gamma, Ad.data_ptr(), n, p, p, X.data_ptr(), p, r,
                                             f.data_ptr(), ev.data_ptr(), 0)
            assert st == spca.SPCA_OK
            torch.cuda.synchronize()
            fh, evh = f.cpu().numpy(), ev.cpu().numpy()
            ref = np.array([oracle.objective(A64, form, gamma, out["start_x"][c].astype(np.float64))
                            for c in range(r)])
            _close(ref[:, 0], fh)
            _close(ref[:, 1], evh)
            _close(out["start_objective"], fh)
            _close(out["start_explained"], evh)
    h.close()
    # a dense x (every column used) and a ragged row count: the coalesced reads cover all of A
    n2, p2, r2 = 517, 2049, 9
    A2 = I.gaussian_matrix(n2, p2, 31).astype(np.float32)
    X2 = I.raw_starts(p2, r2, 32).astype(np.float32)
    A2d, X2d = torch.from_numpy(A2).cuda(), torch.from_numpy(X2).cuda()
    f = torch.zeros(r2, dtype=torch.float64, device="cuda")
    ev = torch.zeros(r2, dtype=torch.float64, device="cuda")
    assert spca.spca_objective_noalloc(8, 0.3, A2d.data_ptr(), n2, p2, p2, X2d.data_ptr(), p2, r2, f.data_ptr(),
                                       ev.data_ptr(), 0) == spca.SPCA_OK
    torch.cuda.synchronize()
    ref = np.array([oracle.objective(A2.astype(np.float64), 8, 0.3, X2[c].astype(np.float64)) for c in range(r2)])
    _close(ref[:, 0], f.cpu().numpy())
    _close(ref[:, 1], ev.cpu().numpy())
    # sizes beyond the fixed scratch are refused before anything runs (A and X are not read: a
    # 2049-row A takes 9 partial pairs per start); so are more than 65535 starts
    n_big = 2049
    r_big = 262144 // ((n_big + 255) // 256) + 1
    assert r_big <= 65535
    st = spca.spca_objective_noalloc(1, 0.0, Ad.data_ptr(), n_big, p, p, Ad.data_ptr(), p, r_big, Ad.data_ptr(),
                                     Ad.data_ptr(), 0)
    assert st == spca.SPCA_E_INVALID
    st = spca.spca_objective_noalloc(1, 0.0, Ad.data_ptr(), 1, p, p, Ad.data_ptr(), p, 65536, Ad.data_ptr(),
                                     Ad.data_ptr(), 0)
    assert st == spca.SPCA_E_UNSUPPORTED
