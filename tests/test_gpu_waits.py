"""Failure detection on the device: every wait inside the tensor-core contraction kernels is
bounded.  With spca_set_waits' test switch the CTA pairs that finish a split tile of the stream-K
schedule wait for a part flag that no CTA ever sets; their waits must run out within the short
limit, the kernel must wind down and return, and the call must report SPCA_E_TIMEOUT.  The
context stays usable: the same handle with normal settings, and a fresh handle, then give the
products of a handle that never timed out."""
import time

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


def _products(lib, h, form, X, r, n, p):
    import torch
    U = torch.zeros((r, n), dtype=torch.float32, device="cuda")
    V = torch.zeros((r, p), dtype=torch.float32, device="cuda")
    st = lib.spca_products(h.h, form, lib.SPCA_ENGINE_TC, X.data_ptr(), p, r, U.data_ptr(), n, V.data_ptr(), p)
    torch.cuda.synchronize()
    return st, U.cpu().numpy(), V.cpu().numpy()


def test_stream_k_wait_runs_out_and_reports_timeout(lib):
    import torch
    # v = A^T y: 32 row tiles of A^T (16 CTA pairs), one 256-wide column tile, 32 K-blocks: the
    # 512 units are split over the resident pairs, so most tiles are finished by an owner that
    # waits for parts of other pairs
    n, p, r = 2048, 4096, 200
    A = I.gaussian_matrix(n, p, 41).astype(np.float32)
    X = torch.from_numpy(I.raw_starts(p, r, 42).astype(np.float32)).cuda()
    ref = lib.Handle(A)
    st, U0, V0 = _products(lib, ref, 1, X, r, n, p)
    assert st == lib.SPCA_OK, lib.spca_last_error(ref.h)

    h = lib.Handle(A)
    h.set_waits(2000, unpublished_parts=True)   # 2 ms, and parts that never come
    t0 = time.perf_counter()
    st, _, _ = _products(lib, h, 1, X, r, n, p)
    dt = time.perf_counter() - t0
    assert st == lib.SPCA_E_TIMEOUT, (st, lib.spca_last_error(h.h))
    assert dt < 1.0, dt                           # bounded by the short limit, not the default 2 s
    # the same handle with normal settings works again, bit for bit
    h.set_waits(2000000, unpublished_parts=False)
    st, U1, V1 = _products(lib, h, 1, X, r, n, p)
    assert st == lib.SPCA_OK, lib.spca_last_error(h.h)
    assert np.array_equal(U1, U0) and np.array_equal(V1, V0)
    h.close()
    # a fresh handle solves as before
    h2 = lib.Handle(A)
    out = h2.solve(1, r, s=20, max_iter=5, tol=-1, x0=X.data_ptr(), x0_device=True, engine=lib.SPCA_ENGINE_TC)
    assert out["objective"] > 0
    h2.close()
    ref.close()


def test_set_waits_rejects_bad_limits(lib):
    A = I.gaussian_matrix(8, 9, 43).astype(np.float32)
    h = lib.Handle(A)
    for us in (0, -5, 60000001):
        assert lib.spca_set_waits(h.h, us, False) == lib.SPCA_E_INVALID
    assert lib.spca_set_waits(None, 1000, False) == lib.SPCA_E_INVALID
    h.close()
