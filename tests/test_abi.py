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


def test_binding_constants_match_the_header():
    """Every integer #define TS_* of the header has the same value in the binding."""
    import re
    import paper_2311_09465_gb300 as ts
    text = open(os.path.join(ROOT, "include", "tsgls.h")).read()
    found = re.findall(r"^#define\s+(TS_\w+)\s+(-?\d+)\b", text, flags=re.M)
    assert len(found) >= 20
    for name, val in found:
        assert getattr(ts, name) == int(val), name


def _c_layout(tmp_path, structs):
    """sizeof and field offsets of the header's structs, from the C compiler."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tsgls.h"', "int main(void) {"]
    for name, fields in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        name, field, val = line.split()
        res[(name, field)] = int(val)
    return res


def test_binding_structs_match_the_header_layout(tmp_path):
    # the ctypes mirrors of ts_params, ts_solve_opts and ts_solve_report have the
    # C header's size and field offsets (a field added on one side only fails here)
    import paper_2311_09465_gb300 as ts
    mirrors = {"ts_params": ts.ts_params, "ts_solve_opts": ts.ts_solve_opts,
               "ts_solve_report": ts.ts_solve_report}
    structs = {name: [f for f, _ in cls._fields_] for name, cls in mirrors.items()}
    c = _c_layout(tmp_path, structs)
    for name, cls in mirrors.items():
        assert c[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert c[(name, f)] == getattr(cls, f).offset, (name, f)
