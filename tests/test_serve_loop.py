"""The request loop's host logic without a GPU: a fake handle and a fake group session stand in for
the C ABI (a solve returns its arguments after a short sleep; a group member finishes after as
many steps as its request asks).  Whole-solve mode: every request gets its own result, requests
run on several workers at once, a worker's clones stay within its memory budget (least recently
used first out), an oversized request is refused, and drain / close finish cleanly.  Group mode:
requests that arrive while a group runs are admitted between its steps, each member leaves with
its own result when it finishes, the members' memory stays within the worker's budget, requests a
group does not take are solved whole by the same worker, and a failed step reaches every member."""
import threading
import time

import pytest

from paper_1212_4137_gb300 import serve


class FakeHandle:
    live = 0
    lock = threading.Lock()
    running = 0
    peak = 0

    def __init__(self, A, stream=0):
        self.n, self.p = A
        self.name = A
        with FakeHandle.lock:
            FakeHandle.live += 1

    def clone(self, stream=0):
        return FakeHandle((self.n, self.p))

    def solve(self, form, r, **kw):
        with FakeHandle.lock:
            FakeHandle.running += 1
            FakeHandle.peak = max(FakeHandle.peak, FakeHandle.running)
        time.sleep(0.01)
        with FakeHandle.lock:
            FakeHandle.running -= 1
        return {"form": form, "r": r, "shape": (self.n, self.p), **kw}

    def close(self):
        with FakeHandle.lock:
            FakeHandle.live -= 1


def _server(**kw):
    kw.setdefault("mode", "solve")
    return serve.Server(handle_factory=FakeHandle, stream_factory=lambda: (None, 0), **kw)


def test_each_request_gets_its_own_result_and_workers_overlap():
    with _server(workers=3, budget_bytes=1 << 34) as s:
        for name, shape in (("a", (100, 500)), ("b", (300, 900)), ("c", (50, 70))):
            s.register(name, shape)
        futs = []
        for i in range(24):
            name = "abc"[i % 3]
            futs.append((name, i, s.submit(name, 1 + i % 8, 4 + i, tag=i)))
        for name, i, f in futs:
            out = f.result(timeout=10)
            assert out["tag"] == i and out["r"] == 4 + i and out["form"] == 1 + i % 8
            assert out["shape"] == {"a": (100, 500), "b": (300, 900), "c": (50, 70)}[name]
            assert out["latency_ms"] >= out["service_ms"] >= 0.0
        s.drain()
    assert FakeHandle.peak >= 2          # solves of different workers overlapped
    assert FakeHandle.live == 0          # every clone and matrix handle closed


def test_memory_budget_evicts_and_refuses():
    one = serve.workspace_bytes(1000, 4000, 64)
    with _server(workers=1, budget_bytes=int(2.5 * one)) as s:
        for name in ("a", "b", "c"):
            s.register(name, (1000, 4000))
        for name in ("a", "b", "c", "a"):
            s.submit(name, 1, 64).result(timeout=10)
        w = s._workers[0]
        assert w.held <= s.worker_budget and len(w.clones) == 2      # the oldest clone was evicted
        assert list(w.clones) == ["c", "a"]
        with pytest.raises(MemoryError):
            s.submit("a", 1, 64 * 10)
        with pytest.raises(KeyError):
            s.submit("zzz", 1, 4)
    assert FakeHandle.live == 0


def test_errors_reach_the_future():
    class Bad(FakeHandle):
        def clone(self, stream=0):
            return Bad((self.n, self.p))

        def solve(self, form, r, **kw):
            raise RuntimeError("solve failed")

    s = serve.Server(workers=2, handle_factory=Bad, stream_factory=lambda: (None, 0), mode="solve")
    s.register("a", (10, 20))
    f = s.submit("a", 1, 4)
    with pytest.raises(RuntimeError):
        f.result(timeout=10)
    s.close()
    with pytest.raises(RuntimeError):
        s.submit("a", 1, 4)


def test_registration_and_configuration_errors():
    with pytest.raises(ValueError):
        _server(workers=0)
    with _server(workers=1, budget_bytes=1 << 30) as s:
        s.register("a", (10, 20))
        with pytest.raises(ValueError):
            s.register("a", (10, 20))
        futs = [s.submit("a", 1, 4, tag=i) for i in range(5)]
        s.drain()                               # returns only when every queued request is done
        assert all(f.done() for f in futs)
        assert [f.result()["tag"] for f in futs] == list(range(5))
    assert FakeHandle.live == 0


# ---------------------------------------------------------------- group mode
class FakeGroup:
    """A group session: a member admitted with kwargs {"steps": k} finishes after k steps."""
    instances = []
    lock = threading.Lock()
    fail_at = None

    def __init__(self, stream=0):
        self.members = {}
        self.steps = 0
        self.admitted_at = {}
        self.max_members = 0
        self.closed = False
        with FakeGroup.lock:
            FakeGroup.instances.append(self)

    def set_tiles(self, tiles):
        self.tiles = tiles

    def admit(self, problems, tags):
        for (h, form, r, kw), tag in zip(problems, tags):
            self.sizes = getattr(self, "sizes", set()) | {serve.request_cost(h.n, h.p, r)}
            self.members[tag] = [kw.get("steps", 1), {"form": form, "r": r, "shape": (h.n, h.p), **kw}]
            self.admitted_at[tag] = self.steps
        self.max_members = max(self.max_members, len(self.members))

    def step(self, sweeps):
        time.sleep(0.005)
        self.steps += 1
        if FakeGroup.fail_at is not None and self.steps >= FakeGroup.fail_at:
            raise RuntimeError("step failed")
        done = []
        for tag, m in list(self.members.items()):
            m[0] -= 1
            if m[0] <= 0:
                done.append((tag, dict(m[1], admitted_at=self.admitted_at[tag], finished_at=self.steps)))
                del self.members[tag]
        return done

    def pending(self):
        return len(self.members)

    def close(self):
        self.closed = True


def _gserver(**kw):
    FakeGroup.instances = []
    FakeGroup.fail_at = None
    return serve.Server(handle_factory=FakeHandle, stream_factory=lambda: (None, 0), group_factory=FakeGroup,
                        mode="group", **kw)


def test_group_mode_admits_between_steps():
    with _gserver(workers=1, budget_bytes=1 << 34) as s:
        s.register("a", (100, 500))
        s.register("b", (300, 900))
        first = s.submit("a", 1, 16, steps=20, tag=0)        # a long request ...
        time.sleep(0.03)
        later = [s.submit("ab"[i % 2], 2, 8, steps=2, tag=1 + i) for i in range(6)]   # ... joined later
        outs = [f.result(timeout=10) for f in later]
        assert not first.done() or first.result()["finished_at"] >= 20
        for i, o in enumerate(outs):
            assert o["tag"] == 1 + i and o["r"] == 8 and o["form"] == 2
            assert o["admitted_at"] >= 1               # admitted while the first request ran
            assert o["finished_at"] - o["admitted_at"] == 2
            assert o["latency_ms"] >= o["service_ms"] >= 0.0
        assert first.result(timeout=10)["finished_at"] == 20
        g = FakeGroup.instances[0]
        assert g.max_members >= 2                      # members swept together
    assert all(g.closed for g in FakeGroup.instances)
    assert FakeHandle.live == 0


def test_group_mode_budget_members_and_whole_solves():
    one = serve.member_bytes(1000, 4000, 64)
    with _gserver(workers=1, budget_bytes=int(2.5 * one), max_members=8) as s:
        s.register("a", (1000, 4000))
        futs = [s.submit("a", 1, 64, steps=3, tag=i) for i in range(5)]
        whole = s.submit("a", 1, 16, lowp_sweeps=4, tag=99)    # not for a group: solved whole
        for f in futs:
            f.result(timeout=10)
        assert whole.result(timeout=10)["tag"] == 99 and "finished_at" not in whole.result()
        assert FakeGroup.instances[0].max_members <= 2      # within the memory budget
        with pytest.raises(MemoryError):
            s.submit("a", 1, 64 * 10)
    assert FakeHandle.live == 0


def test_group_mode_failed_step_reaches_every_member():
    with _gserver(workers=1, budget_bytes=1 << 34) as s:
        FakeGroup.fail_at = 2
        s.register("a", (10, 20))
        futs = [s.submit("a", 1, 4, steps=5, tag=i) for i in range(3)]
        for f in futs:
            with pytest.raises(RuntimeError):
                f.result(timeout=10)
        FakeGroup.fail_at = None
        assert s.submit("a", 1, 4, steps=1, tag=7).result(timeout=10)["tag"] == 7   # the worker goes on


def test_group_mode_size_classes():
    """With size classes each worker's group takes the requests of its class only, so a small
    request never sweeps beside a large one; every request is still served."""
    big = serve.request_cost(3000, 9000, 256)
    with _gserver(workers=2, budget_bytes=1 << 40, classes=[big / 2]) as s:
        s.register("small", (100, 500))
        s.register("large", (3000, 9000))
        futs = [s.submit("small" if i % 3 else "large", 1, 8 if i % 3 else 256, steps=1 + i % 4, tag=i)
                for i in range(30)]
        outs = [f.result(timeout=10) for f in futs]
        assert [o["tag"] for o in outs] == list(range(30))
        used = [g for g in FakeGroup.instances if getattr(g, "sizes", None)]
        assert len(used) == 2
        for g in used:   # one class per group
            assert all(c < big / 2 for c in g.sizes) or all(c >= big / 2 for c in g.sizes)
    with pytest.raises(ValueError):
        _gserver(workers=1, budget_bytes=1 << 30, classes=[1.0])
