"""The C-ABI library builds, loads and exports every entry point include/mls.h declares.

No compute calls: these run without a GPU.
"""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mls.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|int)\s+(mls_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1805_01113_gb300 import build_ext, binding
    build_ext.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("mls_create", "mls_build_transfer", "mls_interpolate", "mls_spread", "mls_marker_prep",
                 "mls_transfer_status", "mls_strerror"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(os.path.join(ROOT, "paper_1805_01113_gb300", "libmls_gb300.so"))
    missing = [n for n in _declared() if not hasattr(raw, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_1805_01113_gb300 import binding
    assert sorted(binding.SIGNATURES) == _declared()


def test_host_only_calls(lib):
    from paper_1805_01113_gb300 import binding as B
    o = B.mls_options()
    assert lib.mls_options_default(ctypes.byref(o)) == B.MLS_OK
    assert (o.real, o.field, o.n_sub, list(o.brick_log2), o.refine) == (B.MLS_F32, B.MLS_F32, 9, [3, 3, 3], 1)
    assert o.eps == 1.0 and o.cond_max == 1e6 and o.basis == 4
    assert lib.mls_options_default(None) == B.MLS_ERR_INVALID_ARG
    assert lib.mls_strerror(B.MLS_ERR_CAPACITY).decode().startswith("more markers")
    # NULL handles are rejected before any CUDA call.
    assert lib.mls_destroy(None) == B.MLS_ERR_INVALID_ARG
    assert lib.mls_build_transfer(None, None, None, None, 0, 0, None) == B.MLS_ERR_INVALID_ARG
    assert lib.mls_create(None, None, None) == B.MLS_ERR_INVALID_ARG
    assert b"NULL" in lib.mls_last_error()


def test_create_rejects_bad_grids_without_gpu(lib):
    from paper_1805_01113_gb300 import binding as B
    g = B.mls_grid()
    faces = [(ctypes.c_double * 5)(0, 1, 2, 3, 4), (ctypes.c_double * 5)(0, 1, 1, 3, 4),
             (ctypes.c_double * 5)(0, 1, 2, 3, 4)]
    for d in range(3):
        g.n[d] = 4
        g.faces[d] = ctypes.cast(faces[d], ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    assert lib.mls_create(ctypes.byref(g), None, ctypes.byref(h)) == B.MLS_ERR_INVALID_ARG
    assert b"increasing" in lib.mls_last_error()
    o = B.mls_options()
    lib.mls_options_default(ctypes.byref(o))
    o.real, o.field = B.MLS_F32, B.MLS_F64
    faces[1] = (ctypes.c_double * 5)(0, 1, 2, 3, 4)
    g.faces[1] = ctypes.cast(faces[1], ctypes.POINTER(ctypes.c_double))
    assert lib.mls_create(ctypes.byref(g), ctypes.byref(o), ctypes.byref(h)) == B.MLS_ERR_INVALID_ARG
    # Only the linear (m = 4) and quadratic (m = 10) bases exist.
    lib.mls_options_default(ctypes.byref(o))
    for m in (0, 3, 7, 11):
        o.basis = m
        assert lib.mls_create(ctypes.byref(g), ctypes.byref(o), ctypes.byref(h)) == B.MLS_ERR_INVALID_ARG
        assert b"basis" in lib.mls_last_error()
