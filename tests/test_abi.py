"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol.

Runs without a GPU: only host-side entry points are called.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "tsgls.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(ts_\w+)\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_09465_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"ts_mesh_load", "ts_residual", "ts_jvp", "ts_solve"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_host_side_validation(lib):
    lib.ts_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.ts_version()
    lib.ts_last_error.restype = ctypes.c_char_p
    xyz = np.zeros((4, 3))
    tets = np.array([[0, 1, 2, 9]], dtype=np.int32)     # node id out of range
    out = ctypes.c_void_p()
    rc = lib.ts_mesh_load(xyz.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(4),
                          tets.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(1),
                          None, None, ctypes.c_int64(0), ctypes.byref(out))
    assert rc == -1 and out.value is None
    assert b"out of range" in lib.ts_last_error()
    rc = lib.ts_residual(None, None, None, ctypes.c_int(64), None)
    assert rc == -1


def test_python_binding_mirrors_the_abi():
    import paper_2311_09465_gb300 as ts
    for n in _declared():
        assert hasattr(ts, n), n
