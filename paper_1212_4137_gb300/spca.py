"""Thin ctypes binding of libspca.so with the names of include/spca.h.

Only argument marshalling lives here: every step of the solve runs in the library's CUDA
kernels.  ``load()`` raises if the library is missing or no GPU is usable; there is no CPU
fallback.  Device buffers are passed as integer addresses (e.g. ``tensor.data_ptr()``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspca.so")

SPCA_OK, SPCA_E_INVALID, SPCA_E_NOMEM, SPCA_E_CUDA, SPCA_E_TIMEOUT, SPCA_E_BUSY, SPCA_E_UNSUPPORTED = range(7)
SPCA_F32, SPCA_F64, SPCA_FP16, SPCA_FP8_E4M3_COLSCALED, SPCA_FP16_RESIDENT = range(5)
SPCA_GAMMA_FIXED, SPCA_GAMMA_TARGET_NNZ = 0, 1
SPCA_ST_MAXITER, SPCA_ST_CONVERGED, SPCA_ST_DEGENERATE = 0, 1, 2
SPCA_ENGINE_AUTO, SPCA_ENGINE_SIMT, SPCA_ENGINE_TC, SPCA_ENGINE_TC_LOWP = 0, 1, 2, 3

# every symbol include/spca.h declares
EXPORTS = ("spca_create", "spca_create_csr", "spca_clone", "spca_solve", "spca_xstep", "spca_products", "spca_deflate", "spca_profile_enable",
           "spca_profile_query", "spca_objective_noalloc", "spca_set_waits",
           "spca_group_create", "spca_group_destroy", "spca_group_last_error", "spca_solve_group",
           "spca_group_set_tiles", "spca_group_admit", "spca_group_step", "spca_group_pending",
           "spca_destroy", "spca_strerror", "spca_last_error")
SPCA_K_ALL, SPCA_K_INIT, SPCA_K_U_DENSE, SPCA_K_U_SPARSE, SPCA_K_YSTEP, SPCA_K_V, SPCA_K_XSTEP, \
    SPCA_K_FINALISE, SPCA_K_PREP = range(-1, 8)
KERNEL_NAMES = {SPCA_K_INIT: "init", SPCA_K_U_DENSE: "u_dense", SPCA_K_U_SPARSE: "u_sparse",
                SPCA_K_YSTEP: "ystep", SPCA_K_V: "v", SPCA_K_XSTEP: "xstep",
                SPCA_K_FINALISE: "finalise", SPCA_K_PREP: "prep"}


class spca_params(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int), ("s", ctypes.c_double), ("gamma", ctypes.c_double),
                ("gamma_mode", ctypes.c_int), ("gamma_calib_sweeps", ctypes.c_int),
                ("r", ctypes.c_int), ("max_iter", ctypes.c_int), ("tol", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("x0_is_device", ctypes.c_int), ("engine", ctypes.c_int),
                ("lowp_sweeps", ctypes.c_int), ("refine_sweeps", ctypes.c_int), ("timeout_us", ctypes.c_int64),
                ("total_starts", ctypes.c_int), ("lowp_first", ctypes.c_int)]


_fp = ctypes.POINTER(ctypes.c_float)
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)


class spca_result(ctypes.Structure):
    _fields_ = [("objective", ctypes.c_double), ("explained_variance", ctypes.c_double),
                ("gamma", ctypes.c_double), ("best_start", ctypes.c_int), ("best_iters", ctypes.c_int),
                ("best_status", ctypes.c_int), ("converged", ctypes.c_int), ("degenerate", ctypes.c_int),
                ("sweeps_total", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("x", _fp), ("y", _fp), ("support", _i64p), ("start_objective", _dp),
                ("start_explained", _dp), ("start_F", _dp), ("start_iters", _ip),
                ("start_status", _ip), ("start_gamma", _dp), ("start_x", _fp)]


class spca_problem(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("prm", spca_params), ("x0", ctypes.c_void_p),
                ("res", ctypes.POINTER(spca_result))]


class spca_group_tiles(ctypes.Structure):
    _fields_ = [("tile_n", ctypes.c_int), ("stages", ctypes.c_int)]


class SpcaError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libspca.so; raises if it is missing (build it with paper_1212_4137_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libspca.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        lib.spca_create.restype = ctypes.c_int
        lib.spca_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_void_p]
        lib.spca_solve.restype = ctypes.c_int
        lib.spca_create_csr.restype = ctypes.c_int
        lib.spca_create_csr.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_void_p]
        lib.spca_clone.restype = ctypes.c_int
        lib.spca_clone.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_void_p]
        lib.spca_solve.argtypes = [ctypes.c_void_p, ctypes.POINTER(spca_params), ctypes.c_void_p,
                                   ctypes.POINTER(spca_result)]
        lib.spca_xstep.restype = ctypes.c_int
        lib.spca_xstep.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                   ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]
        lib.spca_products.restype = ctypes.c_int
        lib.spca_products.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_int64]
        lib.spca_objective_noalloc.restype = ctypes.c_int
        lib.spca_objective_noalloc.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64,
                                               ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                               ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.spca_group_create.restype = ctypes.c_int
        lib.spca_group_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]
        lib.spca_group_destroy.restype = None
        lib.spca_group_destroy.argtypes = [ctypes.c_void_p]
        lib.spca_group_last_error.restype = ctypes.c_char_p
        lib.spca_group_last_error.argtypes = [ctypes.c_void_p]
        lib.spca_solve_group.restype = ctypes.c_int
        lib.spca_solve_group.argtypes = [ctypes.c_void_p, ctypes.POINTER(spca_problem), ctypes.c_int,
                                         ctypes.POINTER(spca_group_tiles)]
        lib.spca_group_set_tiles.restype = ctypes.c_int
        lib.spca_group_set_tiles.argtypes = [ctypes.c_void_p, ctypes.POINTER(spca_group_tiles)]
        lib.spca_group_admit.restype = ctypes.c_int
        lib.spca_group_admit.argtypes = [ctypes.c_void_p, ctypes.POINTER(spca_problem), ctypes.c_int, _ip]
        lib.spca_group_step.restype = ctypes.c_int
        lib.spca_group_step.argtypes = [ctypes.c_void_p, ctypes.c_int, _ip, ctypes.c_int, _ip]
        lib.spca_group_pending.restype = ctypes.c_int
        lib.spca_group_pending.argtypes = [ctypes.c_void_p]
        lib.spca_set_waits.restype = ctypes.c_int
        lib.spca_set_waits.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
        lib.spca_deflate.restype = ctypes.c_int
        lib.spca_deflate.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.spca_profile_enable.restype = ctypes.c_int
        lib.spca_profile_enable.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.spca_profile_query.restype = ctypes.c_int
        lib.spca_profile_query.argtypes = [ctypes.c_void_p, ctypes.c_int, _i64p, _dp]
        lib.spca_destroy.restype = None
        lib.spca_destroy.argtypes = [ctypes.c_void_p]
        lib.spca_strerror.restype = ctypes.c_char_p
        lib.spca_strerror.argtypes = [ctypes.c_int]
        lib.spca_last_error.restype = ctypes.c_char_p
        lib.spca_last_error.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


def spca_strerror(status: int) -> str:
    return load().spca_strerror(int(status)).decode()


def spca_last_error(h) -> str:
    return load().spca_last_error(h).decode()


def _check(status: int, what: str, h=None):
    if status != SPCA_OK:
        detail = spca_last_error(h) if h else ""
        raise SpcaError(status, f"{what} failed: {spca_strerror(status)} {detail}".strip())


def spca_create(A, n: int, p: int, lda: int, in_dtype: int, a_is_device: bool, storage: int = SPCA_F32,
                stream: int = 0):
    """A: host numpy array (C-contiguous) or a device address (int)."""
    h = ctypes.c_void_p()
    ptr = A if isinstance(A, int) else A.ctypes.data
    st = load().spca_create(ctypes.byref(h), ctypes.c_void_p(ptr), n, p, lda, in_dtype,
                            int(a_is_device), storage, ctypes.c_void_p(stream))
    return st, h


def spca_create_csr(n: int, p: int, nnz: int, row_ptr, col_idx, values, is_device: bool, stream: int = 0):
    """row_ptr (int64), col_idx (int32), values (float32): host numpy arrays, or device addresses
    (ints) with is_device."""
    h = ctypes.c_void_p()
    if is_device:
        ptrs = [int(row_ptr), int(col_idx), int(values)]
    else:
        arrs = [np.ascontiguousarray(row_ptr, dtype=np.int64), np.ascontiguousarray(col_idx, dtype=np.int32),
                np.ascontiguousarray(values, dtype=np.float32)]
        ptrs = [a.ctypes.data for a in arrs]
    st = load().spca_create_csr(ctypes.byref(h), int(n), int(p), int(nnz), ctypes.c_void_p(ptrs[0]),
                                ctypes.c_void_p(ptrs[1]), ctypes.c_void_p(ptrs[2]), int(is_device),
                                ctypes.c_void_p(stream))
    return st, h


def spca_solve(h, params: spca_params, x0, result: spca_result) -> int:
    ptr = None if x0 is None else (x0 if isinstance(x0, int) else x0.ctypes.data)
    return load().spca_solve(h, ctypes.byref(params), ctypes.c_void_p(ptr) if ptr else None,
                             ctypes.byref(result))


def spca_xstep(h, form, s, gamma, calibrate, V, ldv, r, X, ldx, F, nnz, thr) -> int:
    return load().spca_xstep(h, int(form), float(s), float(gamma), int(calibrate), ctypes.c_void_p(V),
                             ldv, r, ctypes.c_void_p(X), ldx, ctypes.c_void_p(F), ctypes.c_void_p(nnz),
                             ctypes.c_void_p(thr))


def spca_products(h, form, engine, X, ldx, r, U, ldu, V, ldv) -> int:
    return load().spca_products(h, int(form), int(engine), ctypes.c_void_p(X), ldx, r, ctypes.c_void_p(U), ldu,
                                ctypes.c_void_p(V), ldv)


def spca_objective_noalloc(form, gamma, A, n, p, lda, X, ldx, r, f, ev, stream=0) -> int:
    """All pointers are device addresses (ints)."""
    return load().spca_objective_noalloc(int(form), float(gamma), ctypes.c_void_p(A), n, p, lda,
                                         ctypes.c_void_p(X), ldx, int(r), ctypes.c_void_p(f),
                                         ctypes.c_void_p(ev), ctypes.c_void_p(stream))


def spca_deflate(h, x, x_is_device: bool = False) -> int:
    """x: p floats, a host numpy array or a device address (int)."""
    ptr = x if isinstance(x, int) else np.ascontiguousarray(x, dtype=np.float32).ctypes.data
    keep = None if isinstance(x, int) else np.ascontiguousarray(x, dtype=np.float32)
    if keep is not None:
        ptr = keep.ctypes.data
    return load().spca_deflate(h, ctypes.c_void_p(ptr), int(x_is_device))


def spca_set_waits(h, wait_limit_us: int, unpublished_parts: bool = False) -> int:
    return load().spca_set_waits(h, int(wait_limit_us), int(unpublished_parts))


SPCA_PROFILE_ALL = (1 << 8) - 1


def spca_profile_enable(h, mask: int) -> int:
    return load().spca_profile_enable(h, int(mask))


def spca_profile_query(h, kernel: int):
    """(status, launches, ms)"""
    n = ctypes.c_int64()
    t = ctypes.c_double()
    st = load().spca_profile_query(h, int(kernel), ctypes.byref(n), ctypes.byref(t))
    return st, n.value, t.value


def spca_destroy(h) -> None:
    if h:
        load().spca_destroy(h)


# ------------------------------------------------------------------ convenience wrappers
class Handle:
    """Owns an spca_handle; A is host numpy (float32/float64), a torch CUDA tensor, or a sparse
    matrix (scipy.sparse, or a tuple (indptr, indices, data, (n, p)) of host arrays) kept in
    compressed sparse rows.  storage (dense A): SPCA_F32, SPCA_FP16, SPCA_FP8_E4M3_COLSCALED, or
    SPCA_FP16_RESIDENT (A kept only in 16 bits; every sweep a low-precision one)."""

    def __init__(self, A, stream: int = 0, storage: int = SPCA_F32):
        if isinstance(A, tuple) or hasattr(A, "indptr") or hasattr(A, "tocsr"):
            if isinstance(A, tuple):
                indptr, indices, data, (n, p) = A
            else:
                M = A.tocsr()
                indptr, indices, data, (n, p) = M.indptr, M.indices, M.data, M.shape
            st, h = spca_create_csr(n, p, int(np.asarray(indptr)[-1]), indptr, indices, data, False, stream)
            _check(st, "spca_create_csr")
            self.h, self.n, self.p = h, int(n), int(p)
            return
        try:
            import torch
            is_tensor = isinstance(A, torch.Tensor)
        except ImportError:  # pragma: no cover
            is_tensor = False
        if is_tensor:
            assert A.is_cuda and A.dim() == 2 and A.stride(1) == 1
            dt = {"torch.float32": SPCA_F32, "torch.float64": SPCA_F64}[str(A.dtype)]
            n, p = A.shape
            st, h = spca_create(A.data_ptr(), n, p, A.stride(0), dt, True, storage, stream)
        else:
            A = np.ascontiguousarray(A)
            dt = SPCA_F64 if A.dtype == np.float64 else SPCA_F32
            if A.dtype not in (np.float32, np.float64):
                A = A.astype(np.float32)
            n, p = A.shape
            st, h = spca_create(A, n, p, p, dt, False, storage, stream)
        _check(st, "spca_create")
        self.h, self.n, self.p = h, n, p

    def clone(self, stream: int = 0) -> "Handle":
        """A handle sharing this one's matrix (read-only), with its own stream and workspace."""
        h = ctypes.c_void_p()
        _check(load().spca_clone(ctypes.byref(h), self.h, ctypes.c_void_p(stream)), "spca_clone", self.h)
        other = Handle.__new__(Handle)
        other.h, other.n, other.p = h, self.n, self.p
        return other

    def deflate(self, x, x_device: bool = False):
        """Projection deflation A <- A (I - z z^T), z = x / ||x|| (x: host array or device address)."""
        _check(spca_deflate(self.h, x, x_device), "spca_deflate", self.h)

    def set_waits(self, wait_limit_us: int, unpublished_parts: bool = False):
        """Limit of the tensor-core kernels' device-side waits; unpublished_parts tests its expiry."""
        _check(spca_set_waits(self.h, wait_limit_us, unpublished_parts), "spca_set_waits", self.h)

    def profile(self, on: bool, kernels=None):
        """Time every kernel (on=True), only the given kernel ids, or nothing (on=False)."""
        mask = 0
        if on:
            mask = SPCA_PROFILE_ALL if kernels is None else sum(1 << int(k) for k in set(kernels))
        _check(spca_profile_enable(self.h, mask), "spca_profile_enable", self.h)

    def profile_query(self, kernel: int):
        st, n, ms = spca_profile_query(self.h, kernel)
        _check(st, "spca_profile_query", self.h)
        return n, ms

    def close(self):
        if self.h:
            spca_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, form, r, s=1.0, gamma=0.0, gamma_target=False, calib=10, max_iter=100,
              tol=1e-9, x0=None, seed=0, engine=SPCA_ENGINE_AUTO, want_starts=False, x0_device=False,
              lowp_sweeps=0, refine_sweeps=0, timeout_us=0, total_starts=0, lowp_first=0):
        """Returns a dict of numpy results.  x0: r x p float32 host array, device address
        (x0_device=True), or None for seeded starts."""
        prm = make_params(form, r, s=s, gamma=gamma, gamma_target=gamma_target, calib=calib, max_iter=max_iter,
                          tol=tol, seed=seed, x0_device=x0_device, engine=engine, lowp_sweeps=lowp_sweeps,
                          refine_sweeps=refine_sweeps, timeout_us=timeout_us, total_starts=total_starts,
                          lowp_first=lowp_first)
        nres = max(r, total_starts)
        out, res = _result_buffers(self.n, self.p, nres, want_starts)
        if x0 is not None and not x0_device:
            x0 = np.ascontiguousarray(x0, dtype=np.float32)
            assert x0.shape == (nres, self.p)
        _check(spca_solve(self.h, prm, x0, res), "spca_solve", self.h)
        return _result_dict(out, res)


def make_params(form, r, s=1.0, gamma=0.0, gamma_target=False, calib=10, max_iter=100, tol=1e-9, seed=0,
                x0_device=False, engine=SPCA_ENGINE_AUTO, lowp_sweeps=0, refine_sweeps=0, timeout_us=0,
                total_starts=0, lowp_first=0) -> spca_params:
    return spca_params(form=form, s=s, gamma=gamma,
                       gamma_mode=SPCA_GAMMA_TARGET_NNZ if gamma_target else SPCA_GAMMA_FIXED,
                       gamma_calib_sweeps=calib, r=r, max_iter=max_iter, tol=tol, seed=seed,
                       x0_is_device=int(x0_device), engine=engine, lowp_sweeps=lowp_sweeps,
                       refine_sweeps=refine_sweeps, timeout_us=timeout_us, total_starts=total_starts,
                       lowp_first=lowp_first)


def _result_buffers(n, p, nres, want_starts):
    out = {"x": np.zeros(p, np.float32), "y": np.zeros(n, np.float32), "support": np.zeros(p, np.int64)}
    if want_starts:
        out.update(start_objective=np.zeros(nres), start_explained=np.zeros(nres), start_F=np.zeros(nres),
                   start_iters=np.zeros(nres, np.int32), start_status=np.zeros(nres, np.int32),
                   start_gamma=np.zeros(nres), start_x=np.zeros((nres, p), np.float32))
    res = spca_result()
    for k, v in out.items():
        setattr(res, k, v.ctypes.data_as(type(getattr(res, k))))
    return out, res


def _result_dict(out, res):
    out["support"] = out["support"][:res.nnz]
    for k in ("objective", "explained_variance", "gamma", "best_start", "best_iters", "best_status",
              "converged", "degenerate", "sweeps_total", "nnz"):
        out[k] = getattr(res, k)
    return out


class Group:
    """Owns an spca_group: many problems solved together, each sweep phase one launch over all."""

    def __init__(self, stream: int = 0):
        g = ctypes.c_void_p()
        st = load().spca_group_create(ctypes.byref(g), ctypes.c_void_p(stream))
        _check(st, "spca_group_create")
        self.g = g

    def last_error(self) -> str:
        return load().spca_group_last_error(self.g).decode()

    def _problems(self, problems, want_starts):
        """The C array for `problems` and, per problem, its result buffers and the host arrays that
        must outlive the call."""
        count = len(problems)
        arr = (spca_problem * count)()
        entries = []
        for i, (h, form, r, kw) in enumerate(problems):
            kw = dict(kw)
            x0 = kw.pop("x0", None)
            ws = kw.pop("want_starts", want_starts)
            prm = make_params(form, r, **kw)
            out, res = _result_buffers(h.n, h.p, r, ws)
            keep = [res]
            if x0 is not None and not prm.x0_is_device:
                x0 = np.ascontiguousarray(x0, dtype=np.float32)
                assert x0.shape == (r, h.p)
                keep.append(x0)
                x0p = x0.ctypes.data
            else:
                x0p = x0
            arr[i].h = h.h
            arr[i].prm = prm
            arr[i].x0 = x0p
            arr[i].res = ctypes.pointer(res)
            entries.append((out, res, keep))
        return arr, entries

    def _fail(self, st, what):
        raise SpcaError(st, f"{what} failed: {spca_strerror(st)} {self.last_error()}")

    def solve(self, problems, tiles=None, want_starts=False):
        """problems: list of (Handle, form, r, kwargs) with the keyword arguments of Handle.solve
        (x0: host array or device address with x0_device=True).  tiles: (tile_n, stages), "auto"
        (the measured shape of tuning.py's table) or None (the library's default).
        Returns one result dict per problem, as Handle.solve does."""
        arr, entries = self._problems(problems, want_starts)
        if tiles == "auto":   # the measured shape for this mix's bucket (tuning.py), else the default
            from . import tuning
            tiles = tuning.choose(max(r for _, _, r, _ in problems))
        t = spca_group_tiles(*(tiles or (0, 0)))
        st = load().spca_solve_group(self.g, arr, len(problems), ctypes.byref(t))
        if st != SPCA_OK:
            self._fail(st, "spca_solve_group")
        return [_result_dict(out, res) for out, res, _ in entries]

    # ---- the group as a session: admit problems while others run, step their sweeps
    def set_tiles(self, tiles=None):
        t = spca_group_tiles(*(tiles or (0, 0)))
        st = load().spca_group_set_tiles(self.g, ctypes.byref(t))
        if st != SPCA_OK:
            self._fail(st, "spca_group_set_tiles")

    def admit(self, problems, tags, want_starts=False):
        """Admit problems (as for solve) under integer tags; their results come back from step()."""
        arr, entries = self._problems(problems, want_starts)
        tg = (ctypes.c_int * len(tags))(*tags)
        st = load().spca_group_admit(self.g, arr, len(problems), tg)
        if st != SPCA_OK:
            self._fail(st, "spca_group_admit")
        if not hasattr(self, "_held"):
            self._held = {}
        for t, e in zip(tags, entries):
            self._held[int(t)] = e

    def step(self, sweeps: int = 4):
        """Run `sweeps` sweeps of every member; returns [(tag, result dict)] of the members that
        finished."""
        cap = max(1, self.pending())
        fin = (ctypes.c_int * cap)()
        nf = ctypes.c_int(0)
        st = load().spca_group_step(self.g, int(sweeps), fin, cap, ctypes.byref(nf))
        if st != SPCA_OK:
            self._fail(st, "spca_group_step")
        done = []
        for i in range(min(nf.value, cap)):
            out, res, _ = self._held.pop(int(fin[i]))
            done.append((int(fin[i]), _result_dict(out, res)))
        return done

    def pending(self) -> int:
        return int(load().spca_group_pending(self.g))

    def close(self):
        if getattr(self, "g", None):
            load().spca_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
