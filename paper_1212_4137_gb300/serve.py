"""A request loop over the C ABI: resident matrices, memory-bounded admission, and solves of
different requests running at the same time on one GPU.

Matrices are registered once (``spca_create`` / ``spca_create_csr``: copied to the device and kept
there).  Workers, each a host thread with its own CUDA stream, take requests in arrival order; a
worker solves on a clone of the request's matrix (``spca_clone``: the matrix shared read-only,
the clone's own stream, workspace and captured graphs).  The solves of different workers overlap
on the device, so a request that arrives while others run starts as soon as a worker and memory
are free: continuous batching at the granularity of whole solves.

Admission by memory: every worker keeps its clones (their workspaces and graphs make repeated
requests on a matrix cheap) within ``budget_bytes / workers``; a request whose workspace estimate
does not fit evicts the worker's least recently used clones first, and a request larger than a
worker's whole budget is refused.  The estimate is the handle's per-solve workspace for (n, p, r).

Each solve is a deterministic function of its own inputs (fixed-order reductions, no schedule
dependence), so a request's result is the same alone and in the mix.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time
from dataclasses import dataclass, field

from . import spca


def workspace_bytes(n: int, p: int, r: int) -> int:
    """Device bytes a handle's per-solve workspace takes for r starts (an upper estimate): x, v,
    u, y and their 16-bit planes, support lists, candidate lists, per-start scalars, the union
    operands and the packed operand of the sparse products."""
    pn, pp = (n + 7) // 8 * 8, (p + 7) // 8 * 8
    per_start = 4 * (2 * pp + 2 * pn) + 2 * 2 * (pp + pn) + 8 * pp + 8 * 1024 + 4 * max(pn, pp) + 256
    return int(r * per_start + 2 * 2 * pn * 1024 + (1 << 20))


@dataclass
class Request:
    name: str
    form: int
    r: int
    kwargs: dict
    future: cf.Future
    t_submit: float = field(default_factory=time.perf_counter)
    t_start: float = 0.0
    t_end: float = 0.0


class _Worker:
    def __init__(self, server: "Server", index: int):
        self.server = server
        self.index = index
        self.clones: "collections.OrderedDict[str, tuple]" = collections.OrderedDict()   # name -> (handle, bytes)
        self.held = 0
        self.stream = None
        self.thread = threading.Thread(target=self._run, name=f"spca-worker-{index}", daemon=True)

    def _clone(self, name: str, need: int):
        s = self.server
        if name in self.clones:
            h, b = self.clones.pop(name)
            self.held -= b
        else:
            h = s._base[name].clone(stream=self.stream_ptr)
            b = 0
        # keep the clone's workspace within this worker's budget: drop least recently used clones
        b = max(b, need)
        while self.clones and self.held + b > s.worker_budget:
            _, (old, ob) = self.clones.popitem(last=False)
            old.close()
            self.held -= ob
        self.clones[name] = (h, b)
        self.held += b
        return h

    def _run(self):
        s = self.server
        self.stream, self.stream_ptr = s._stream_factory()
        while True:
            req = s._next()
            if req is None:
                break
            try:
                n, p = s._shape[req.name]
                h = self._clone(req.name, workspace_bytes(n, p, max(req.r, req.kwargs.get("total_starts", 0))))
                req.t_start = time.perf_counter()
                out = h.solve(req.form, req.r, **req.kwargs)
                req.t_end = time.perf_counter()
                out["queue_ms"] = 1e3 * (req.t_start - req.t_submit)
                out["service_ms"] = 1e3 * (req.t_end - req.t_start)
                out["latency_ms"] = 1e3 * (req.t_end - req.t_submit)
                out["worker"] = self.index
                req.future.set_result(out)
            except Exception as e:   # reported through the request's future
                req.future.set_exception(e)
            finally:
                s._done(req)
        for h, _ in self.clones.values():
            h.close()
        self.clones.clear()


class Server:
    """Resident matrices and `workers` concurrent solvers (see the module docstring)."""

    def __init__(self, workers: int = 4, budget_bytes: int = 32 << 30, device: int = 0, handle_factory=None,
                 stream_factory=None):
        """handle_factory(A, stream=...) makes a matrix's handle (spca.Handle); stream_factory() gives
        a worker (stream object, cudaStream_t as int) on the calling thread (a new CUDA stream on
        `device`).  Both are replaceable for tests of the loop without a GPU."""
        if workers < 1:
            raise ValueError("workers must be >= 1")
        self.device = device
        self._handle_factory = handle_factory or spca.Handle
        self._stream_factory = stream_factory or self._cuda_stream
        self.worker_budget = budget_bytes // workers
        self._base = {}
        self._shape = {}
        self._queue: "collections.deque[Request]" = collections.deque()
        self._cv = threading.Condition()
        self._closing = False
        self._in_flight = 0
        self._workers = [_Worker(self, i) for i in range(workers)]
        for w in self._workers:
            w.thread.start()

    def _cuda_stream(self):
        import torch
        torch.cuda.set_device(self.device)
        st = torch.cuda.Stream()
        return st, st.cuda_stream

    def register(self, name: str, A, stream: int = 0) -> None:
        """Copy a matrix to the device (dense array or tensor, or a sparse matrix / CSR tuple)."""
        if name in self._base:
            raise ValueError(f"matrix {name!r} is already registered")
        h = self._handle_factory(A, stream=stream)
        self._base[name] = h
        self._shape[name] = (h.n, h.p)

    def submit(self, name: str, form: int, r: int, **kwargs) -> cf.Future:
        """Queue a solve (the arguments of Handle.solve); the future gives its result dict, with the
        request's queue, service and total latency in ms."""
        if self._closing:
            raise RuntimeError("the server is closed")
        if name not in self._base:
            raise KeyError(f"no matrix {name!r}")
        n, p = self._shape[name]
        if workspace_bytes(n, p, max(r, kwargs.get("total_starts", 0))) > self.worker_budget:
            raise MemoryError(f"a solve of {r} starts on {name!r} exceeds a worker's memory budget")
        fut: cf.Future = cf.Future()
        with self._cv:
            if self._closing:
                raise RuntimeError("the server is closed")
            self._queue.append(Request(name, form, r, dict(kwargs), fut))
            self._cv.notify()
        return fut

    def _next(self):
        with self._cv:
            while not self._queue and not self._closing:
                self._cv.wait()
            if not self._queue:
                return None
            self._in_flight += 1
            return self._queue.popleft()

    def _done(self, req: Request) -> None:
        with self._cv:
            self._in_flight -= 1
            self._cv.notify_all()

    def drain(self) -> None:
        """Wait until every queued request has finished."""
        with self._cv:
            while self._queue or self._in_flight:
                self._cv.wait()

    def close(self) -> None:
        with self._cv:
            self._closing = True
            self._cv.notify_all()
        for w in self._workers:
            w.thread.join()
        for h in self._base.values():
            h.close()
        self._base.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
