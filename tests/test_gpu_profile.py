"""The measurement hooks with graph-replayed sweeps: per-kernel launch counts and event timings
are charged at every replay of a captured segment, timing only the selected kernels, and the
results of a profiled solve are those of an unprofiled one (bit for bit)."""
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


@pytest.mark.parametrize("kernels", [None, "v"])
def test_profiled_solve_matches_and_counts(lib, kernels):
    n, p, r = 400, 1800, 64
    A = I.spiked_matrix(n, p, I.spiked_thetas(n, p), 20, 61, dtype=np.float32)
    G = I.raw_starts(p, r, 62).astype(np.float32)
    h = lib.Handle(A)
    # the per-sweep kernels (AUTO would run this small matrix in one launch per solve)
    kw = dict(s=20.0, x0=G, max_iter=40, tol=1e-7, want_starts=True, engine=lib.SPCA_ENGINE_SIMT)
    plain = h.solve(3, r, **kw)
    h.profile(True, kernels=None if kernels is None else (lib.SPCA_K_V,))
    prof = h.solve(3, r, **kw)
    counts = {k: h.profile_query(k) for k in lib.KERNEL_NAMES}
    total, _ = h.profile_query(lib.SPCA_K_ALL)
    h.profile(False)
    h.close()
    assert np.array_equal(plain["start_x"], prof["start_x"])
    assert prof["objective"] == plain["objective"]
    sweeps = int(prof["start_iters"].max())
    n_v, ms_v = counts[lib.SPCA_K_V]
    # one v = A^T y per queued sweep, replays included; sweeps are queued 4 at a time, so up to 3
    # more than the longest start ran may be queued (their kernels find no active start)
    assert sweeps <= n_v <= sweeps + 3
    assert ms_v > 0.0
    assert total == sum(c[0] for c in counts.values())
    for k, (nl, ms) in counts.items():
        if kernels == "v" and k != lib.SPCA_K_V:
            assert ms == 0.0                   # only the selected kernel is timed
        if nl == 0:
            assert ms == 0.0
