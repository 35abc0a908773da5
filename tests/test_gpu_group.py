"""Groups of problems (spca_solve_group): many independent problems drawn like the batching
configuration (spiked models of random size, a random formulation and s per problem, 64 starts
each) solved together, every sweep phase one launch over all of them.  Each problem must give what
it gives alone (spca_solve on its handle) and what the FP64 oracle gives, at the parity tests'
tolerances; repeating a group solve (graphs replayed) gives the same bits; bad problems are refused."""
import numpy as np
import pytest

from paper_1212_4137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

OBJ_RTOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1212_4137_gb300 import build, spca
    build.build()
    spca.load()
    return spca


def _draw(count, seed, n_range=(150, 1200), p_range=(400, 5000)):
    """Problems like the batching configuration, smaller: n, p log-uniform, 3 spikes of 20 nonzeros,
    a uniform formulation and s in [5, 40] (the gamma-targeting rule for the penalties)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        p = int(round(np.exp(rng.uniform(np.log(p_range[0]), np.log(p_range[1])))))
        form = int(rng.integers(1, 9))
        s = int(min(p, rng.integers(5, 41)))
        A = I.spiked_matrix(n, p, I.spiked_thetas(n, p, (40.0, 30.0, 20.0)), 20, 5000 + seed * 100 + i,
                            dtype=np.float32)
        kw = dict(s=float(s)) if form <= 4 else dict(s=float(s), gamma_target=True, calib=5)
        out.append((A, form, kw))
    return out


def test_group_matches_solo_and_oracle(lib, oracle):
    probs = _draw(12, 1)
    r, sweeps = 64, 25
    handles = [lib.Handle(A) for A, _, _ in probs]
    starts = [I.raw_starts(A.shape[1], r, 600 + i).astype(np.float32) for i, (A, _, _) in enumerate(probs)]
    g = lib.Group()
    req = [(h, form, r, dict(kw, x0=G, max_iter=sweeps, tol=-1)) for h, (A, form, kw), G in zip(handles, probs, starts)]
    outs = g.solve(req, want_starts=True)
    again = g.solve(req, want_starts=True)   # replayed graphs: the same bits
    for o, a in zip(outs, again):
        assert np.array_equal(o["start_x"], a["start_x"]) and o["objective"] == a["objective"]
    for i, ((A, form, kw), h, G, o) in enumerate(zip(probs, handles, starts, outs)):
        solo = h.solve(form, r, x0=G, max_iter=sweeps, tol=-1, want_starts=True, engine=lib.SPCA_ENGINE_TC, **kw)
        assert np.array_equal(o["start_iters"], solo["start_iters"]), i
        close = np.abs(o["start_objective"] - solo["start_objective"]) <= OBJ_RTOL * np.maximum(
            1.0, np.abs(solo["start_objective"]))
        dx = np.abs(o["start_x"] - solo["start_x"]).max(axis=1)
        assert np.mean(close & (dx <= 1e-4)) >= 0.95, (i, form, np.mean(close), dx.max())
        assert abs(o["objective"] - solo["objective"]) <= OBJ_RTOL * max(1.0, abs(solo["objective"])), i
        ref = oracle.solve(A.astype(np.float64), form, G.astype(np.float64), max_iter=sweeps, tol=-1, **kw)
        assert abs(o["objective"] - ref.f[ref.best]) <= OBJ_RTOL * max(1.0, abs(ref.f[ref.best])), (i, form)
        mo = np.abs(o["start_objective"] - ref.f) <= OBJ_RTOL * np.maximum(1.0, np.abs(ref.f))
        mx = np.abs(o["start_x"] - ref.X).max(axis=1) <= 1e-4
        assert np.mean(mo & mx) >= 0.95, (i, form, np.mean(mo & mx))
        # the outputs of the best start
        b = o["best_start"]
        assert np.array_equal(o["support"], np.flatnonzero(o["start_x"][b]))
    g.close()
    for h in handles:
        h.close()


def test_group_stopping_rule_and_seeded_starts(lib):
    probs = _draw(6, 2)
    r = 40
    handles = [lib.Handle(A) for A, _, _ in probs]
    g = lib.Group()
    req = [(h, form, r, dict(kw, seed=77, max_iter=200, tol=1e-6)) for h, (A, form, kw) in zip(handles, probs)]
    outs = g.solve(req, want_starts=True, tiles=(128, 2))
    for (A, form, kw), h, o in zip(probs, handles, outs):
        solo = h.solve(form, r, seed=77, max_iter=200, tol=1e-6, want_starts=True, engine=lib.SPCA_ENGINE_TC, **kw)
        # a start's stopping sweep can move by a few sweeps with the rounding (see the single-solve
        # stopping-rule test); the best objective agrees
        assert abs(o["objective"] - solo["objective"]) <= 1e-4 * max(1.0, abs(solo["objective"]))
        assert np.mean(np.abs(o["start_iters"] - solo["start_iters"]) <= 3) >= 0.75
        assert np.all(o["start_iters"] <= 200)
    g.close()
    for h in handles:
        h.close()


def test_group_rejects_bad_problems(lib):
    A = I.gaussian_matrix(50, 80, 3).astype(np.float32)
    h = lib.Handle(A)
    g = lib.Group()
    for bad in (dict(s=100.0), dict(s=5.0, lowp_sweeps=2), dict(s=5.0, total_starts=99)):
        with pytest.raises(lib.SpcaError) as e:
            g.solve([(h, 1, 8, bad)])
        assert e.value.status == lib.SPCA_E_INVALID
    with pytest.raises(lib.SpcaError) as e:
        g.solve([(h, 1, 8, dict(s=5.0))], tiles=(96, 3))
    assert e.value.status == lib.SPCA_E_INVALID
    ip, ix, v = I.bag_of_words(40, 60, 300, 4)
    hs = lib.Handle((ip, ix, v, (40, 60)))
    with pytest.raises(lib.SpcaError) as e:
        g.solve([(hs, 1, 8, dict(s=5.0))])
    assert e.value.status == lib.SPCA_E_INVALID and "dense" in g.last_error()
    # a good problem after the refusals still solves
    out = g.solve([(h, 1, 8, dict(s=5.0, seed=3, max_iter=10))])[0]
    assert out["objective"] > 0
    g.close()
    h.close()
    hs.close()


def test_group_session_admits_while_others_run(lib):
    """Continuous batching at sweep boundaries: problems admitted at different times into a running
    group sweep in the same launches as the others; each problem's result is bit for bit its result
    alone (a group of one), whatever else is in the mix."""
    probs = _draw(9, 3)
    r = 32
    handles = [lib.Handle(A) for A, _, _ in probs]
    kws = [dict(kw, seed=500 + i, max_iter=[12, 30, 60][i % 3], tol=1e-7 if i % 2 else -1)
           for i, (A, form, kw) in enumerate(probs)]
    alone = []
    g1 = lib.Group()
    for h, (A, form, _), kw in zip(handles, probs, kws):
        alone.append(g1.solve([(h, form, r, kw)], want_starts=True)[0])
    g1.close()
    g = lib.Group()
    done = {}
    waves = [[0, 1, 2], [3, 4], [5], [6, 7, 8]]
    for wave in waves:
        g.admit([(handles[i], probs[i][1], r, kws[i]) for i in wave], wave, want_starts=True)
        for tag, out in g.step(4):
            done[tag] = out
    while g.pending():
        for tag, out in g.step(4):
            done[tag] = out
    assert sorted(done) == list(range(len(probs)))
    for i, out in done.items():
        assert np.array_equal(out["start_x"], alone[i]["start_x"]), i
        assert np.array_equal(out["start_iters"], alone[i]["start_iters"]), i
        assert out["objective"] == alone[i]["objective"] and out["best_start"] == alone[i]["best_start"], i
    g.close()
    for h in handles:
        h.close()


def test_group_pools_match_alone(lib, oracle):
    """Members on one matrix share v = A^T y (a pool: their active starts side by side in one
    operand, the matrix read once per sweep for all of them).  Each member's results are still its
    results alone, bit for bit, whatever the other members' active counts put its starts at, and
    members of another plane type (y = +-1) on the same matrix take their own pool."""
    n, p = 900, 3100
    A = I.spiked_matrix(n, p, I.spiked_thetas(n, p, (40.0, 30.0, 20.0)), 20, 6100, dtype=np.float32)
    h = lib.Handle(A)
    reqs = [(h, 1, 16, dict(seed=11, s=20.0, max_iter=30, tol=1e-7)),
            (h, 3, 40, dict(seed=12, s=20.0, max_iter=50, tol=-1)),
            (h, 2, 24, dict(seed=13, s=20.0, max_iter=40, tol=1e-7)),
            (h, 5, 7, dict(seed=14, s=20.0, gamma_target=True, calib=6, max_iter=45, tol=1e-7)),
            (h, 4, 70, dict(seed=15, s=20.0, max_iter=25, tol=1e-7))]
    g = lib.Group()
    alone = [g.solve([q], want_starts=True)[0] for q in reqs]
    together = g.solve(reqs, want_starts=True)
    for i, (a, t) in enumerate(zip(alone, together)):
        assert np.array_equal(a["start_x"], t["start_x"]), i
        assert np.array_equal(a["start_iters"], t["start_iters"]), i
        assert a["objective"] == t["objective"], i
    # and admitted at different times into a running session
    done = {}
    for wave in ([0, 2], [1], [3, 4]):
        g.admit([reqs[i] for i in wave], wave, want_starts=True)
        for tag, out in g.step(4):
            done[tag] = out
    while g.pending():
        for tag, out in g.step(4):
            done[tag] = out
    for i, out in done.items():
        assert np.array_equal(out["start_x"], alone[i]["start_x"]), i
    g.close()
    # the pooled solve against the oracle on one member
    A64 = A.astype(np.float64)
    G = I.raw_starts(p, 40, 12)   # not the seeded starts: a fresh solve with given starts
    g = lib.Group()
    outs = g.solve([(h, 3, 40, dict(x0=G.astype(np.float32), s=20.0, max_iter=30, tol=-1)),
                    (h, 1, 16, dict(seed=11, s=20.0, max_iter=30, tol=1e-7))], want_starts=True)
    g.close()
    ref = oracle.solve(A64, 3, G.astype(np.float32).astype(np.float64), s=20.0, max_iter=30, tol=-1)
    close = np.abs(outs[0]["start_objective"] - ref.f) <= OBJ_RTOL * np.maximum(1.0, np.abs(ref.f))
    assert np.mean(close) >= 0.95
    h.close()


def test_group_seeded_starts_are_the_solo_starts(lib):
    """A group sets up its members' starts in its own launch (in their first sweep): seeded starts
    are the ones spca_solve draws for the same seed, and given starts are normalised the same way,
    so after one sweep each start's x agrees with the solo solve's to the contraction's rounding."""
    probs = _draw(4, 7)
    r = 24
    handles = [lib.Handle(A) for A, _, _ in probs]
    g = lib.Group()
    req = [(h, form, r, dict(kw, seed=900 + i, max_iter=1, tol=-1)) for i, (h, (A, form, kw)) in
           enumerate(zip(handles, probs))]
    outs = g.solve(req, want_starts=True)
    g.close()
    for (h, form, r_, kw), o in zip(req, outs):
        solo = h.solve(form, r_, want_starts=True, engine=lib.SPCA_ENGINE_TC, **kw)
        dx = np.abs(o["start_x"] - solo["start_x"]).max(axis=1)
        assert np.mean(dx <= 1e-4) >= 0.95, (form, dx.max())
    for h in handles:
        h.close()
