"""The request loop's host logic without a GPU: a fake handle stands in for the C ABI (its solve
returns its arguments after a short sleep).  Every request gets its own result, requests run on
several workers at once, a worker's clones stay within its memory budget (least recently used
first out), an oversized request is refused, and drain / close finish cleanly."""
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

    s = serve.Server(workers=2, handle_factory=Bad, stream_factory=lambda: (None, 0))
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
