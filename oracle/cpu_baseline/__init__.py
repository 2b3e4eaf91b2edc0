"""CPU timing baseline of the same algorithm as the GPU library (qgcpu.c):
radix-2 FFT, Lanczos minimal-residual solves, implicit midpoint with the
carried H psi, Suzuki composition, FP64, OpenMP over wavepackets.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): bench.py times it as the
same-algorithm CPU baseline and the tests pin it to the dense oracle.  It
shares no code with the CUDA library.
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "qgcpu.c")
LIB = os.path.join(HERE, "libqgcpu.so")
_lib = None


def build(force=False):
    """Compile qgcpu.c with gcc and OpenMP (skipped when up to date)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-fcx-limited-range", "-std=c11", "-D_GNU_SOURCE",
           "-o", LIB + ".tmp", SRC, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("gcc failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(LIB + ".tmp", LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P, I, D, Lg = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
        L.qgcpu_propagate.restype = I
        L.qgcpu_propagate.argtypes = [I, D, D, I, D, P, P, P, I, I, D, Lg, D, I, ctypes.POINTER(I),
                                      ctypes.POINTER(Lg), ctypes.POINTER(Lg)]
        _lib = L
    return _lib


def propagate(psi, qmin, qmax, mass, V, F, order, dt, nsteps, tol=1e-15, max_iters=600):
    """Propagate packets psi (npk, S, N) complex128 in place by nsteps composed
    implicit-midpoint steps (Suzuki order `order`, step dt).  Returns a dict
    with the status, thread count and H psi / iteration totals."""
    psi = np.asarray(psi)
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    npk, S, n = psi.shape
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    th, hp, it = ctypes.c_int(), ctypes.c_long(), ctypes.c_long()
    st = _load().qgcpu_propagate(n, qmin, qmax, S, mass, V.ctypes.data, F.ctypes.data, psi.ctypes.data, npk, order,
                                 dt, nsteps, tol, max_iters, ctypes.byref(th), ctypes.byref(hp), ctypes.byref(it))
    return {"status": st, "threads": th.value, "hpsi": hp.value, "iters": it.value}
