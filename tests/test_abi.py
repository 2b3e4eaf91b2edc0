"""The C-ABI library builds, loads and exports every symbol include/qgeom.h
declares; host-only entry points answer without a GPU."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qgeom.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qg_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(qglib):
    declared = _declared()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", qglib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (qg_\w+)", out))
    assert set(declared) <= exported, sorted(set(declared) - exported)
    assert sorted(qglib.EXPORTED) == declared
    for name in declared:
        assert hasattr(qglib.lib(), name)


def test_host_only_entry_points(qglib):
    L = qglib.lib()
    assert b"qgeom" in L.qg_version()
    assert L.qg_status_string(2) == b"implicit solve did not converge"
    o = qglib.default_solver_opts()
    assert (o.tol, o.restart, o.max_iters, o.reorth) == (1e-12, 30, 400, 1)
    h = ctypes.c_void_p()
    n = (ctypes.c_int * 1)(100)
    lo = (ctypes.c_double * 1)(0.0)
    hi = (ctypes.c_double * 1)(1.0)
    assert L.qg_create_grid(1, n, lo, hi, ctypes.byref(h)) == qglib.QG_ERR_INVALID_ARG
    assert L.qg_create_grid(3, n, lo, hi, ctypes.byref(h)) == qglib.QG_ERR_INVALID_ARG
    assert L.qg_propagate(None, 0, 2, 0, 1.0, 1, None, None) == qglib.QG_ERR_INVALID_ARG
