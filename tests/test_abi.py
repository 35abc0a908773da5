"""CPU-side checks of the boundary: the library builds for sm_103a, loads, and exports every
symbol include/spca.h declares; the ctypes structures match the header's field order; and
without a GPU the calls fail loudly instead of falling back to the CPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spca.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spca_[a-z_0-9]+)\s*\(", text)))


def _struct_fields(name):
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", text).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            m = re.search(r"\**\s*([A-Za-z_][A-Za-z_0-9]*)\s*(\[\d+\])?\s*$", part.strip())
            fields.append(m.group(1))
    return fields


@pytest.fixture(scope="module")
def lib():
    from paper_1212_4137_gb300 import build, spca
    build.build()
    return spca


def test_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert set(declared) == set(lib.EXPORTS)
    so = lib.load()
    for name in declared:
        assert hasattr(so, name), name


def test_struct_layout_matches_header(lib):
    assert [f for f, _ in lib.spca_params._fields_] == _struct_fields("spca_params")
    assert [f for f, _ in lib.spca_result._fields_] == _struct_fields("spca_result")


def _enum_values(names):
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for name in names:
        m = re.search(r"\b" + name + r"\s*=\s*(-?\d+)", text)
        out[name] = int(m.group(1))
    return out


def test_constants_match_header(lib):
    kids = ("SPCA_K_ALL", "SPCA_K_INIT", "SPCA_K_U_DENSE", "SPCA_K_U_SPARSE", "SPCA_K_YSTEP", "SPCA_K_V",
            "SPCA_K_XSTEP", "SPCA_K_FINALISE", "SPCA_K_PREP", "SPCA_K_COUNT")
    vals = _enum_values(kids)
    for name in kids[:-1]:
        assert getattr(lib, name) == vals[name], name
    assert lib.SPCA_PROFILE_ALL == (1 << vals["SPCA_K_COUNT"]) - 1
    text = open(HEADER).read()
    assert "#define SPCA_PROFILE_ALL ((1 << SPCA_K_COUNT) - 1)" in text
    m = re.search(r"#define SPCA_NOALLOC_MAX_PARTIALS (\d+)", text)
    assert m and int(m.group(1)) == 262144


def test_enums_and_group_structs_match_header(lib):
    names = ("SPCA_OK", "SPCA_E_INVALID", "SPCA_E_NOMEM", "SPCA_E_CUDA", "SPCA_E_TIMEOUT", "SPCA_E_BUSY",
             "SPCA_E_UNSUPPORTED", "SPCA_F32", "SPCA_F64", "SPCA_FP16", "SPCA_FP8_E4M3_COLSCALED",
             "SPCA_FP16_RESIDENT", "SPCA_ST_MAXITER", "SPCA_ST_CONVERGED", "SPCA_ST_DEGENERATE",
             "SPCA_ENGINE_AUTO", "SPCA_ENGINE_SIMT", "SPCA_ENGINE_TC", "SPCA_ENGINE_TC_LOWP")
    vals = _enum_values(names)
    for name in names:
        assert getattr(lib, name) == vals[name], name
    assert [f for f, _ in lib.spca_problem._fields_] == _struct_fields("spca_problem")
    assert [f for f, _ in lib.spca_group_tiles._fields_] == _struct_fields("spca_group_tiles")


def test_strerror_is_static_text(lib):
    assert lib.spca_strerror(0) == "ok"
    assert lib.spca_strerror(1) == "invalid argument"
    assert lib.spca_strerror(12345) == "unknown status"


def test_bad_arguments_rejected_before_device(lib):
    so = lib.load()
    h = ctypes.c_void_p()
    A = np.zeros((2, 3), np.float32)
    for (n, p, lda, dt) in ((0, 3, 3, 0), (2, 0, 3, 0), (2, 3, 2, 0), (2, 3, 3, 7)):
        st = so.spca_create(ctypes.byref(h), ctypes.c_void_p(A.ctypes.data), n, p, lda, dt, 0, 0, None)
        assert st == lib.SPCA_E_INVALID
    st = so.spca_create(ctypes.byref(h), None, 2, 3, 3, 0, 0, 0, None)
    assert st == lib.SPCA_E_INVALID
    st = so.spca_create(ctypes.byref(h), ctypes.c_void_p(A.ctypes.data), 2, 3, 3, 0, 0, lib.SPCA_F64, None)
    assert st == lib.SPCA_E_UNSUPPORTED     # FP64 storage is not built
    st = so.spca_create(ctypes.byref(h), ctypes.c_void_p(A.ctypes.data), 2, 3, 3, 0, 0, 9, None)
    assert st == lib.SPCA_E_INVALID
    # a dense A's rows ride on a grid dimension in blocks of 256 (at most 65535 blocks); A is not read
    st = so.spca_create(ctypes.byref(h), ctypes.c_void_p(A.ctypes.data), 65535 * 256 + 1, 1, 1, 0, 0, 0, None)
    assert st == lib.SPCA_E_UNSUPPORTED
    f = np.zeros(4)
    so.spca_objective_noalloc.restype = ctypes.c_int
    for r, want in ((65536, lib.SPCA_E_UNSUPPORTED), (0, lib.SPCA_E_INVALID)):
        st = so.spca_objective_noalloc(1, ctypes.c_double(0.0), ctypes.c_void_p(A.ctypes.data), ctypes.c_int64(2),
                                       ctypes.c_int64(3), ctypes.c_int64(3), ctypes.c_void_p(A.ctypes.data),
                                       ctypes.c_int64(3), r, ctypes.c_void_p(f.ctypes.data),
                                       ctypes.c_void_p(f.ctypes.data), None)
        assert st == want, r
    assert so.spca_solve(None, None, None, None) == lib.SPCA_E_INVALID
    assert so.spca_profile_enable(None, 1) == lib.SPCA_E_INVALID
    so.spca_set_waits.restype = ctypes.c_int
    assert so.spca_set_waits(None, ctypes.c_int64(1000), 0) == lib.SPCA_E_INVALID
    so.spca_destroy(None)


def test_no_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, h = lib.spca_create(np.zeros((2, 3), np.float32), 2, 3, 3, lib.SPCA_F32, False)
    assert st == lib.SPCA_E_CUDA
