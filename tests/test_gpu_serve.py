"""Clones and the request loop on the GPU.

spca_clone shares a matrix read-only: a clone's solve matches the FP64 oracle like any handle's,
the matrix outlives the handle it came from, and deflation of a shared matrix is refused.  The
request loop runs solves of different requests at the same time; each request's result must be
the same alone (one worker, one request at a time) and in the mix (four workers, every request
queued at once), bit for bit, since a solve depends only on its own inputs.  The same holds in
group mode, where requests join running group sessions between sweep segments and sweep in the
same launches as the other members."""
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


def test_clone_shares_the_matrix(lib, oracle):
    n, p, r = 400, 1500, 40
    A = I.spiked_matrix(n, p, I.spiked_thetas(n, p), 20, 31, dtype=np.float32)
    G = I.raw_starts(p, r, 32).astype(np.float32)
    h = lib.Handle(A)
    c1 = h.clone()
    c2 = c1.clone()
    with pytest.raises(lib.SpcaError) as e:       # the matrix is shared
        h.deflate(np.ones(p, np.float32))
    assert e.value.status == lib.SPCA_E_UNSUPPORTED
    h.close()                                      # the clones keep the matrix
    ref = oracle.solve(A.astype(np.float64), 3, G.astype(np.float64), s=20.0, max_iter=100, tol=1e-9)
    for c in (c1, c2):
        for eng in (lib.SPCA_ENGINE_TC, lib.SPCA_ENGINE_SIMT):
            out = c.solve(3, r, s=20.0, x0=G, max_iter=100, tol=1e-9, engine=eng)
            assert abs(out["objective"] - ref.f[ref.best]) <= 1e-5 * ref.f[ref.best]
    c1.close()
    c2.deflate(G[0])                               # the last holder may deflate
    c2.close()


def _requests(rng, names, shapes, count):
    reqs = []
    for i in range(count):
        name = names[i % len(names)]
        n, p = shapes[name]
        form = int(rng.integers(1, 9))
        s = float(min(int(rng.integers(5, 40)), p))
        r = int(rng.choice([1, 16, 64]))
        kw = dict(s=s, seed=1000 + i, max_iter=60, tol=1e-9, want_starts=True)
        if form >= 5:
            kw.update(gamma_target=True, calib=6)
        reqs.append((name, form, r, kw))
    return reqs


def test_requests_same_alone_and_in_the_mix(lib):
    from paper_1212_4137_gb300 import serve
    rng = np.random.default_rng(33)
    mats = {}
    for k, (n, p) in enumerate([(300, 1200), (800, 2500), (150, 600)]):
        mats[f"d{k}"] = I.spiked_matrix(n, p, I.spiked_thetas(n, p), 15, 40 + k, dtype=np.float32)
    ip, ix, v = I.bag_of_words(700, 1500, 15000, 44)
    shapes = {name: A.shape for name, A in mats.items()}
    shapes["bow"] = (700, 1500)
    reqs = _requests(rng, list(shapes), shapes, 24)

    def run(workers, one_at_a_time, mode):
        outs = []
        with serve.Server(workers=workers, budget_bytes=8 << 30, mode=mode) as s:
            for name, A in mats.items():
                s.register(name, A)
            s.register("bow", (ip, ix, v, (700, 1500)))
            if one_at_a_time:
                for q in reqs:
                    outs.append(s.submit(q[0], q[1], q[2], **q[3]).result())
            else:
                futs = [s.submit(q[0], q[1], q[2], **q[3]) for q in reqs]
                outs = [f.result() for f in futs]
        return outs

    for mode in ("solve", "group"):
        alone = run(1, True, mode)
        mixed = run(4 if mode == "solve" else 2, False, mode)
        assert len({o["worker"] for o in mixed}) > 1   # (group mode: each worker's group held several)
        for a, m in zip(alone, mixed):
            assert a["objective"] == m["objective"]
            assert a["best_start"] == m["best_start"] and a["sweeps_total"] == m["sweeps_total"]
            assert np.array_equal(a["x"], m["x"]) and np.array_equal(a["start_x"], m["start_x"])
            assert np.array_equal(a["start_objective"], m["start_objective"])
        if mode == "group":
            # a group's results agree with whole solves at the parity tolerances
            whole = run(1, True, "solve")
            close = [abs(a["objective"] - w["objective"]) <= 1e-4 * max(1.0, abs(w["objective"]))
                     for a, w in zip(alone, whole)]
            assert np.mean(close) >= 0.9
