"""ctypes wrapper around the FP64 CPU oracle (``spca_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` are the only callers.  The product path (``paper_1212_4137_gb300``) never
imports this module.

All arrays are float64; A is n x p row-major, or a scipy.sparse matrix (kept in compressed
sparse rows: the products of Algorithm 2 run over the stored entries and give the dense
result); starts and iterates are stored one per row (r x p).  Formulation numbers follow
Table 1 of the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spca_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ST_MAXITER, ST_CONVERGED, ST_DEGENERATE = 0, 1, 2

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-O2, OpenMP over starts)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_lambda_s.restype = ctypes.c_double
        lib.oracle_lambda_s.argtypes = [_dp, ctypes.c_int64, ctypes.c_double]
        for name in ("oracle_op_T",):
            getattr(lib, name).argtypes = [_dp, ctypes.c_int64, ctypes.c_int64, _dp]
        for name in ("oracle_op_U", "oracle_op_V"):
            getattr(lib, name).argtypes = [_dp, ctypes.c_int64, ctypes.c_double, _dp]
        lib.oracle_xstep.restype = ctypes.c_int
        lib.oracle_xstep.argtypes = [ctypes.c_int, _dp, ctypes.c_int64, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, _dp, _dp, _i64p, _dp]
        lib.oracle_objective.argtypes = [_dp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                         ctypes.c_double, _dp, _dp, _dp]
        lib.oracle_solve.restype = ctypes.c_int
        lib.oracle_solve.argtypes = [_dp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                     _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     _dp, _dp, _dp, _dp, _ip, _ip, _dp, _dp, ctypes.c_int]
        lib.oracle_objective_csr.argtypes = [_i64p, _ip, _dp, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
        lib.oracle_solve_csr.restype = ctypes.c_int
        lib.oracle_solve_csr.argtypes = [_i64p, _ip, _dp] + lib.oracle_solve.argtypes[1:]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _c(a: np.ndarray, dtype=np.float64) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp if a.dtype == np.float64 else (_ip if a.dtype == np.int32 else _i64p))


def _csr(A):
    """(indptr int64, indices int32, data float64, n, p) of a scipy.sparse matrix in canonical
    compressed sparse rows (columns ascending within a row, repeated entries summed), or None
    for a dense array."""
    if not hasattr(A, "tocsr"):
        return None
    M = A.tocsr(copy=True)
    M.sum_duplicates()
    M.sort_indices()
    n, p = M.shape
    return (_c(M.indptr, np.int64), _c(M.indices, np.int32), _c(M.data), n, p)


def num_threads() -> int:
    return _load().oracle_num_threads()


def op_T(a, s: int) -> np.ndarray:
    a = _c(a); z = np.empty_like(a)
    _load().oracle_op_T(_p(a), a.size, int(s), _p(z)); return z


def op_U(a, gamma: float) -> np.ndarray:
    a = _c(a); z = np.empty_like(a)
    _load().oracle_op_U(_p(a), a.size, float(gamma), _p(z)); return z


def op_V(a, gamma: float) -> np.ndarray:
    a = _c(a); z = np.empty_like(a)
    _load().oracle_op_V(_p(a), a.size, float(gamma), _p(z)); return z


def lambda_s(a, s: float) -> float:
    a = _c(a)
    return _load().oracle_lambda_s(_p(a), a.size, float(s))


@dataclass
class XStep:
    x: np.ndarray
    F: float
    nnz: int
    thr: float
    degenerate: bool


def xstep(form: int, v, s: float, gamma: float = 0.0, calibrate: bool = False) -> XStep:
    """One x-step of Algorithm 2 on v (normalised x, Table 3 value, nnz, threshold)."""
    v = _c(v); x = np.empty_like(v)
    F = ctypes.c_double(); nnz = ctypes.c_int64(); thr = ctypes.c_double()
    deg = _load().oracle_xstep(int(form), _p(v), v.size, float(s), float(gamma), int(calibrate),
                               _p(x), ctypes.byref(F), ctypes.byref(nnz), ctypes.byref(thr))
    return XStep(x, F.value, nnz.value, thr.value, bool(deg))


def objective(A, form: int, gamma: float, x):
    """(f(x) of Table 1, explained variance) in FP64."""
    x = _c(x); f = ctypes.c_double(); ev = ctypes.c_double()
    sp = _csr(A)
    if sp is not None:
        ptr, col, val, n, p = sp
        _load().oracle_objective_csr(_p(ptr), _p(col), _p(val), n, p, int(form), float(gamma),
                                     _p(x), ctypes.byref(f), ctypes.byref(ev))
    else:
        A = _c(A)
        _load().oracle_objective(_p(A), A.shape[0], A.shape[1], int(form), float(gamma), _p(x),
                                 ctypes.byref(f), ctypes.byref(ev))
    return f.value, ev.value


@dataclass
class Solve:
    best: int
    X: np.ndarray        # r x p final iterates
    f: np.ndarray        # Table 1 objective per start
    ev: np.ndarray       # explained variance per start
    F: np.ndarray        # last F value per start
    iters: np.ndarray    # sweeps per start
    status: np.ndarray   # ST_* per start
    gamma: np.ndarray    # gamma used per start (penalty forms)
    F_hist: np.ndarray   # r x max_iter, NaN past the last sweep


def solve(A, form: int, G, s: float = 1.0, gamma: float = 0.0, gamma_target: bool = False,
          calib: int = 10, max_iter: int = 100, tol: float = 1e-9, nthreads: int = 0) -> Solve:
    """Algorithm 2 from the raw starts G (r x p, one per row; normalised inside)."""
    G = _c(G)
    sp = _csr(A)
    if sp is not None:
        ptr, col, val, n, p = sp
        mat = (_p(ptr), _p(col), _p(val))
        entry = _load().oracle_solve_csr
    else:
        A = _c(A)
        n, p = A.shape
        mat = (_p(A),)
        entry = _load().oracle_solve
    r = G.shape[0]
    assert G.shape[1] == p
    X = np.empty((r, p)); f = np.empty(r); ev = np.empty(r); F = np.empty(r)
    iters = np.empty(r, np.int32); status = np.empty(r, np.int32); gam = np.empty(r)
    F_hist = np.empty((r, max(max_iter, 1)))
    best = entry(*mat, n, p, int(form), float(s), float(gamma), int(gamma_target), int(calib),
                 _p(G), r, int(max_iter), float(tol), _p(X), _p(f), _p(ev), _p(F), _p(iters),
                 _p(status), _p(gam), _p(F_hist), int(nthreads))
    return Solve(best, X, f, ev, F, iters, status, gam, F_hist[:, :max_iter])


def deflate(A, x):
    """Projection deflation for a further component: A (I - z z^T) with z = x / ||x||_2, in FP64.

    The paper computes several components (Section 1) but leaves the deflation scheme open;
    projection deflation removes the direction z from every row of A, so that z (and anything
    it dominated) cannot be found again, and keeps A positive semidefinite as A^T A."""
    A = np.asarray(A, dtype=np.float64)
    z = np.asarray(x, dtype=np.float64)
    z = z / np.linalg.norm(z)
    return A - np.outer(A @ z, z)
