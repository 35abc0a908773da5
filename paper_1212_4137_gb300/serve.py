"""A request loop over the C ABI: resident matrices, memory-bounded admission, and solves of
different requests running at the same time on one GPU.

Two modes.  In ``group`` mode (the default) each worker owns a group session (``spca.Group``):
between segments of ``sweeps_per_step`` sweeps it admits the requests waiting in the queue into the
group, whose members all sweep in the same launches (every phase of a sweep one launch over all
members), and the requests whose starts have all stopped leave the group with their results --
continuous batching at sweep boundaries.  Requests a group does not take (a sparse matrix,
low-precision sweeps, on-the-fly replacement) are solved whole by the same worker between two
segments.  In ``solve`` mode each request is one whole solve on a clone of its matrix (below).

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
dependence), and a group member's result does not depend on the other members, so a request's
result is the same alone and in the mix.
"""
from __future__ import annotations

import bisect
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


def member_bytes(n: int, p: int, r: int) -> int:
    """Device bytes of a group member's block (an upper estimate): x, v, u and their 16-bit planes,
    support lists, per-start scalars, the finalisation's partial sums and outputs."""
    pn, pp = (n + 7) // 8 * 8, (p + 7) // 8 * 8
    per_start = 4 * (2 * pp + pn) + 2 * 2 * (pp + pn) + 8 * pp + 16 * ((n + 255) // 256) + 128
    return int(r * per_start + 16 * (pp + pn) + 4096)


def request_cost(n: int, p: int, r: int) -> float:
    """A request's size for the size classes: the multiply-adds of one sweep's v = A^T y with the
    starts padded by one 64-wide tile (a contraction over few starts still reads all of A)."""
    return float(n) * float(p) * float(r + 64)


def groupable(kwargs: dict, sparse: bool) -> bool:
    """Whether a group session takes the request (dense matrix, FP32 sweeps from r starts)."""
    return (not sparse and not kwargs.get("lowp_sweeps") and kwargs.get("total_starts", 0) <= 0
            and kwargs.get("engine", spca.SPCA_ENGINE_AUTO) in (spca.SPCA_ENGINE_AUTO, spca.SPCA_ENGINE_TC))


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
    group_bytes: object = None   # a group member's bytes, or None for a whole solve
    cls: int = 0                 # its size class (group mode with classes)


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

    def _solve_whole(self, req: "Request"):
        s = self.server
        try:
            n, p = s._shape[req.name]
            h = self._clone(req.name, workspace_bytes(n, p, max(req.r, req.kwargs.get("total_starts", 0))))
            req.t_start = time.perf_counter()
            out = h.solve(req.form, req.r, **req.kwargs)
            req.t_end = time.perf_counter()
            self._deliver(req, out)
        except Exception as e:   # reported through the request's future
            req.future.set_exception(e)
        finally:
            s._done(req)

    def _deliver(self, req: "Request", out: dict) -> None:
        out["queue_ms"] = 1e3 * (req.t_start - req.t_submit)
        out["service_ms"] = 1e3 * (req.t_end - req.t_start)
        out["latency_ms"] = 1e3 * (req.t_end - req.t_submit)
        out["worker"] = self.index
        req.future.set_result(out)

    def _run(self):
        s = self.server
        self.stream, self.stream_ptr = s._stream_factory()
        if s.mode == "group":
            self._run_group()
        else:
            while True:
                req = s._next()
                if req is None:
                    break
                self._solve_whole(req)
        for h, _ in self.clones.values():
            h.close()
        self.clones.clear()

    def _run_group(self):
        """Admit waiting requests between segments, step the group, deliver the finished ones."""
        s = self.server
        g = s._group_factory(self.stream_ptr)
        if s.tiles:
            g.set_tiles(s.tiles)
        members = {}   # tag -> (request, bytes)
        held = 0
        tag = 0
        try:
            while True:
                batch = s._take(block=not members, budget=s.worker_budget - held, have=len(members),
                                max_members=s.max_members, cls=self.index % (len(s.classes) + 1))
                if batch is None:
                    break
                admit = []
                for req in batch:
                    if req.group_bytes is None:      # not for a group: a whole solve now
                        self._solve_whole(req)
                        continue
                    req.t_start = time.perf_counter()
                    tag += 1
                    members[tag] = (req, req.group_bytes)
                    held += req.group_bytes
                    admit.append((tag, req))
                if admit:
                    try:
                        g.admit([(s._base[r.name], r.form, r.r, r.kwargs) for _, r in admit], [t for t, _ in admit])
                    except Exception as e:
                        for t, r in admit:
                            members.pop(t)
                            held -= r.group_bytes
                            r.future.set_exception(e)
                            s._done(r)
                if not members:
                    continue
                try:
                    finished = g.step(s.sweeps_per_step)
                except Exception as e:   # the whole group fails: report it to every member
                    for t, (r, b) in list(members.items()):
                        r.future.set_exception(e)
                        s._done(r)
                    members.clear()
                    held = 0
                    g.close()
                    g = s._group_factory(self.stream_ptr)
                    continue
                now = time.perf_counter()
                for t, out in finished:
                    req, b = members.pop(t)
                    held -= b
                    req.t_end = now
                    self._deliver(req, out)
                    s._done(req)
        finally:
            g.close()


class Server:
    """Resident matrices and `workers` concurrent solvers (see the module docstring)."""

    def __init__(self, workers: int = 4, budget_bytes: int = 32 << 30, device: int = 0, handle_factory=None,
                 stream_factory=None, mode: str = "group", sweeps_per_step: int = 4, max_members: int = 1024,
                 tiles=None, group_factory=None, classes=None):
        """handle_factory(A, stream=...) makes a matrix's handle (spca.Handle); stream_factory() gives
        a worker (stream object, cudaStream_t as int) on the calling thread (a new CUDA stream on
        `device`); group_factory(stream) makes a worker's group session (spca.Group).  All three
        are replaceable for tests of the loop without a GPU.  mode: "group" (sessions, continuous
        batching at sweep boundaries) or "solve" (whole solves on clones).  tiles: the grouped
        contraction's tile shape, (tile_n, stages) or None.  classes: in group mode, ascending
        thresholds on a request's size (request_cost: n p (r + 64)) that split the requests into
        len(classes) + 1 classes; worker i serves class i mod (len(classes) + 1) only, so that a
        small request sweeps beside other small ones (a group's sweep lasts as long as all its
        members' work).  Needs at least that many workers."""
        if workers < 1:
            raise ValueError("workers must be >= 1")
        self.classes = sorted(float(c) for c in (classes or ()))
        if mode == "group" and len(self.classes) + 1 > workers:
            raise ValueError("need at least one worker per size class")
        if mode not in ("group", "solve"):
            raise ValueError("mode must be 'group' or 'solve'")
        self.mode = mode
        self.sweeps_per_step = sweeps_per_step
        self.max_members = max_members
        self.tiles = tiles
        self._group_factory = group_factory or (lambda stream: spca.Group(stream=stream))
        self._sparse = {}
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

    def register(self, name: str, A, stream: int = 0, **handle_kwargs) -> None:
        """Copy a matrix to the device (dense array or tensor, or a sparse matrix / CSR tuple);
        handle_kwargs go to the handle factory (e.g. storage=spca.SPCA_FP16_RESIDENT: the matrix
        kept only in 16 bits)."""
        if name in self._base:
            raise ValueError(f"matrix {name!r} is already registered")
        h = self._handle_factory(A, stream=stream, **handle_kwargs)
        self._base[name] = h
        self._shape[name] = (h.n, h.p)
        self._sparse[name] = isinstance(A, tuple) and len(A) == 4 or hasattr(A, "indptr") or hasattr(A, "tocsr")

    def submit(self, name: str, form: int, r: int, **kwargs) -> cf.Future:
        """Queue a solve (the arguments of Handle.solve); the future gives its result dict, with the
        request's queue, service and total latency in ms."""
        if self._closing:
            raise RuntimeError("the server is closed")
        if name not in self._base:
            raise KeyError(f"no matrix {name!r}")
        n, p = self._shape[name]
        gb = None
        if self.mode == "group" and groupable(kwargs, self._sparse.get(name, False)):
            gb = member_bytes(n, p, r)
            need = gb
        else:
            need = workspace_bytes(n, p, max(r, kwargs.get("total_starts", 0)))
        if need > self.worker_budget:
            raise MemoryError(f"a solve of {r} starts on {name!r} exceeds a worker's memory budget")
        fut: cf.Future = cf.Future()
        with self._cv:
            if self._closing:
                raise RuntimeError("the server is closed")
            req = Request(name, form, r, dict(kwargs), fut)
            req.group_bytes = gb
            req.cls = bisect.bisect_left(self.classes, request_cost(n, p, r)) if self.mode == "group" else 0
            self._queue.append(req)
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

    def _take(self, block: bool, budget: int, have: int, max_members: int, cls: int = 0):
        """For a group worker of size class `cls`: the waiting requests of that class, in arrival
        order, that fit the worker's remaining memory and member count (requests not for a group
        count nothing); blocks while there are none if `block`.  None when the server closes and
        the worker has nothing left."""
        nclass = len(self.classes) + 1
        mine = (lambda q: q.cls == cls) if nclass > 1 else (lambda q: True)
        with self._cv:
            while block and not self._closing and not any(mine(q) for q in self._queue):
                self._cv.wait()
            waiting = [q for q in self._queue if mine(q)]
            if not waiting:
                return None if (self._closing and block) else []
            # at most an even share of the class's queue per worker of the class, so that idle
            # workers take the rest
            peers = sum(1 for w in self._workers if w.index % nclass == cls)
            share = max(1, -(-len(waiting) // peers))
            out = []
            for req in waiting:
                if len(out) >= share:
                    break
                gb = req.group_bytes or 0
                if req.group_bytes is not None and (gb > budget or have + 1 > max_members):
                    break
                out.append(req)
                self._in_flight += 1
                if req.group_bytes is not None:
                    budget -= gb
                    have += 1
            if out:
                taken = set(map(id, out))
                self._queue = collections.deque(q for q in self._queue if id(q) not in taken)
            return out

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
