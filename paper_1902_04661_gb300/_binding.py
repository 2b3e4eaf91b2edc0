"""Thin ctypes binding of libqgeom (include/qgeom.h).

Argument marshalling only: every step of the propagation runs in the CUDA
library.  Functions keep the C names (qg_create_grid, qg_propagate, ...);
Grid / Model / State are small owners of the handles for Python callers.
Host data are numpy arrays; device data are torch CUDA tensors (their
data_ptr and the current torch stream are passed through).

If libqgeom.so is missing the import of this module succeeds but every call
raises QgLibraryMissing: there is no fallback path.
"""
import ctypes
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libqgeom.so")

QG_OK = 0
QG_ERR_INVALID_ARG = 1
QG_ERR_NOT_CONVERGED = 2
QG_ERR_CUDA = 3
QG_ERR_OOM = 4
QG_ERR_TIMEOUT = 5
QG_ERR_UNSUPPORTED = 6
QG_TRAPEZOIDAL = 0
QG_MIDPOINT = 1
QG_EXPLICIT_EULER = 2
QG_IMPLICIT_EULER = 3
QG_SOD = 4
QG_TRIPLE_JUMP = 0
QG_SUZUKI = 1
QG_OPTIMAL = 2
QG_C128 = 0
QG_C64_MIXED = 1
QG_SOLVER_GMRES = 0
QG_SOLVER_LANCZOS = 1
QG_GUESS_EULER = 0
QG_GUESS_ZERO = 1
QG_RUN_FORWARD = 0
QG_RUN_CHECKPOINT = 1
QG_RUN_ADJOINT = 2

# Every symbol declared in include/qgeom.h.
EXPORTED = [
    "qg_default_solver_opts", "qg_create_grid", "qg_destroy_grid", "qg_create_model",
    "qg_create_model_diabatic", "qg_model_fields", "qg_destroy_model", "qg_create_state",
    "qg_destroy_state", "qg_state_set_stream", "qg_set_state", "qg_get_state", "qg_set_gaussian",
    "qg_apply_h", "qg_step_implicit", "qg_propagate", "qg_norm", "qg_energy", "qg_population",
    "qg_overlap", "qg_batch_propagate", "qg_batch_create", "qg_batch_run", "qg_batch_capture", "qg_batch_replay", "qg_batch_stats",
    "qg_batch_stream", "qg_batch_destroy", "qg_batch_autotune", "qg_batch_tuning", "qg_selftest_barrier_timeout", "qg_state_set_launch_width",
    "qg_state_autotune", "qg_state_set_adjoint", "qg_propagate_ex", "qg_batch_run_ex", "qg_propagate_noalloc", "qg_status_string", "qg_last_error_string", "qg_version",
    "qg_state_set_cluster", "qg_cluster_size", "qg_batch_cluster", "qg_batch_set_cluster",
    "qg_create_model_diabatic_rep", "qg_diabatic_to_adiabatic", "qg_adiabatic_to_diabatic", "qg_interpolate",
    "qg_batch_classes", "qg_probe_fp64",
]


class QgLibraryMissing(ImportError):
    pass


class QgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


class SolverOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("reorth", ctypes.c_int), ("midpoint_epilogue", ctypes.c_int), ("true_residual", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int), ("solver", ctypes.c_int),
                ("guess", ctypes.c_int)]


class StepStats(ctypes.Structure):
    _fields_ = [("n_hpsi", ctypes.c_int64), ("n_krylov", ctypes.c_int64), ("n_substeps", ctypes.c_int64),
                ("max_krylov", ctypes.c_int32), ("status", ctypes.c_int32), ("max_residual", ctypes.c_double),
                ("failed_step", ctypes.c_int64), ("n_ortho", ctypes.c_int64), ("n_update", ctypes.c_int64),
                ("n_restart", ctypes.c_int64), ("n_hpsi32", ctypes.c_int64), ("n_outer", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """The loaded library (raises QgLibraryMissing if it was never built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise QgLibraryMissing("libqgeom.so not found at %s: run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
        PP = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "qg_default_solver_opts": (V, [ctypes.POINTER(SolverOpts)]),
            "qg_create_grid": (I, [I, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(D), PP]),
            "qg_destroy_grid": (V, [P]),
            "qg_create_model": (I, [P, I, ctypes.POINTER(D), P, P, I, PP]),
            "qg_create_model_diabatic": (I, [P, I, ctypes.POINTER(D), P, P, I, PP]),
            "qg_model_fields": (I, [P, P, P, I]),
            "qg_destroy_model": (V, [P]),
            "qg_create_state": (I, [P, I, PP]),
            "qg_destroy_state": (V, [P]),
            "qg_state_set_stream": (I, [P, P]),
            "qg_set_state": (I, [P, P, I]),
            "qg_get_state": (I, [P, P, I]),
            "qg_set_gaussian": (I, [P, I, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)]),
            "qg_apply_h": (I, [P, P, I]),
            "qg_step_implicit": (I, [P, I, I, I, D, ctypes.POINTER(SolverOpts), ctypes.POINTER(StepStats)]),
            "qg_propagate": (I, [P, I, I, I, D, ctypes.c_int64, ctypes.POINTER(SolverOpts),
                                 ctypes.POINTER(StepStats)]),
            "qg_norm": (I, [P, ctypes.POINTER(D)]),
            "qg_energy": (I, [P, ctypes.POINTER(D)]),
            "qg_population": (I, [P, ctypes.POINTER(D)]),
            "qg_overlap": (I, [P, P, ctypes.POINTER(D)]),
            "qg_batch_propagate": (I, [ctypes.POINTER(P), I, I, I, I, D, ctypes.c_int64,
                                       ctypes.POINTER(SolverOpts), ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(StepStats)]),
            "qg_batch_create": (I, [ctypes.POINTER(P), I, PP]),
            "qg_batch_run": (I, [P, I, I, I, D, ctypes.c_int64, ctypes.POINTER(SolverOpts),
                                 ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(StepStats)]),
            "qg_batch_capture": (I, [P, I, I, I, D, ctypes.c_int64, ctypes.POINTER(SolverOpts)]),
            "qg_batch_replay": (I, [P]),
            "qg_batch_stats": (I, [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(StepStats)]),
            "qg_batch_stream": (P, [P]),
            "qg_batch_autotune": (I, [P, I, I, I, D, ctypes.c_int64, ctypes.POINTER(SolverOpts),
                                      ctypes.POINTER(ctypes.c_double)]),
            "qg_batch_tuning": (I, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
            "qg_selftest_barrier_timeout": (I, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
            "qg_state_set_launch_width": (I, [P, I]),
            "qg_state_set_cluster": (I, [P, I]),
            "qg_create_model_diabatic_rep": (I, [P, I, ctypes.POINTER(D), P, I, PP]),
            "qg_diabatic_to_adiabatic": (I, [P, P, P, I]),
            "qg_adiabatic_to_diabatic": (I, [P, P, P, I]),
            "qg_interpolate": (I, [P, P]),
            "qg_probe_fp64": (I, [ctypes.POINTER(D)] * 5),
            "qg_batch_classes": (I, [P, ctypes.POINTER(I)] + [ctypes.POINTER(I)] * 5),
            "qg_cluster_size": (I, [I, I, I]),
            "qg_batch_cluster": (I, [P, ctypes.POINTER(ctypes.c_int)]),
            "qg_batch_set_cluster": (I, [P, I]),
            "qg_state_autotune": (I, [P, I, I, I, D, ctypes.c_int64, ctypes.POINTER(SolverOpts),
                                      ctypes.POINTER(ctypes.c_double)]),
            "qg_batch_destroy": (V, [P]),
            "qg_state_set_adjoint": (I, [P, P, ctypes.c_int64, ctypes.c_int64, P, P, P]),
            "qg_propagate_ex": (I, [P, I, I, I, I, D, ctypes.c_int64, ctypes.POINTER(SolverOpts),
                                    ctypes.POINTER(StepStats)]),
            "qg_batch_run_ex": (I, [P, I, I, I, I, D, ctypes.c_int64, ctypes.POINTER(SolverOpts),
                                    ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(StepStats)]),
            "qg_propagate_noalloc": (I, [I, D, D, I, D, P, P, P, I, I, I, D, ctypes.c_int64,
                                         ctypes.POINTER(SolverOpts), ctypes.POINTER(StepStats), P]),
            "qg_status_string": (ctypes.c_char_p, [I]),
            "qg_last_error_string": (ctypes.c_char_p, []),
            "qg_version": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st, what, allow=()):
    if st != QG_OK and st not in allow:
        L = lib()
        msg = "%s: %s" % (what, L.qg_status_string(st).decode())
        if st == QG_ERR_CUDA:
            msg += " [%s]" % L.qg_last_error_string().decode()
        raise QgError(st, msg)
    return st


def _dbl_array(vals):
    vals = [float(v) for v in vals]
    return (ctypes.c_double * len(vals))(*vals)


def _host_or_device(x, dtype):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.is_cuda:
                if not x.is_contiguous():
                    raise ValueError("device tensors must be contiguous")
                want = torch.complex128 if dtype == np.complex128 else torch.float64
                if x.dtype != want:
                    raise ValueError("device tensor must be %s" % want)
                return ctypes.c_void_p(x.data_ptr()), 1, x
            x = x.numpy()
    except ImportError:
        pass
    a = np.ascontiguousarray(x, dtype=dtype)
    return ctypes.c_void_p(a.ctypes.data), 0, a


def default_solver_opts(**kw):
    o = SolverOpts()
    lib().qg_default_solver_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def qg_create_grid(N, qmin, qmax):
    D = len(N)
    h = ctypes.c_void_p()
    _check(lib().qg_create_grid(D, (ctypes.c_int * D)(*N), _dbl_array(qmin), _dbl_array(qmax), ctypes.byref(h)),
           "qg_create_grid")
    return h


def qg_create_model(grid, S, mass, V, F):
    h = ctypes.c_void_p()
    pv, dv, kv = _host_or_device(V, np.float64)
    pf, df, kf = _host_or_device(F, np.float64)
    if dv != df:
        raise ValueError("V and F must both be host or both be device buffers")
    _check(lib().qg_create_model(grid, S, _dbl_array(mass), pv, pf, dv, ctypes.byref(h)), "qg_create_model")
    return h


def qg_create_model_diabatic(grid, S, mass, W, dW):
    h = ctypes.c_void_p()
    pw, dw, kw = _host_or_device(W, np.float64)
    pd, dd, kd = _host_or_device(dW, np.float64)
    if dw != dd:
        raise ValueError("W and dW must both be host or both be device buffers")
    _check(lib().qg_create_model_diabatic(grid, S, _dbl_array(mass), pw, pd, dw, ctypes.byref(h)),
           "qg_create_model_diabatic")
    return h


def qg_create_state(model, precision=QG_C128):
    h = ctypes.c_void_p()
    _check(lib().qg_create_state(model, precision, ctypes.byref(h)), "qg_create_state")
    return h


class Grid:
    def __init__(self, N, qmin, qmax):
        self.N = [int(n) for n in N]
        self.qmin = [float(v) for v in qmin]
        self.qmax = [float(v) for v in qmax]
        self.D = len(self.N)
        self.dq = [(b - a) / n for a, b, n in zip(self.qmin, self.qmax, self.N)]
        self.ntot = int(np.prod(self.N))
        self.handle = qg_create_grid(self.N, self.qmin, self.qmax)

    def points(self, d=0):
        return self.qmin[d] + self.dq[d] * np.arange(self.N[d])

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qg_destroy_grid(self.handle)
            self.handle = None


class Model:
    """Adiabatic model from V, F or from a diabatic W with dW (Sec. II E), or,
    with representation="diabatic", the diabatic-representation model of W."""

    def __init__(self, grid, S, mass, V=None, F=None, W=None, dW=None, representation="adiabatic"):
        self.grid = grid
        self.S = int(S)
        self.mass = [float(m) for m in mass]
        self.representation = representation
        if representation == "diabatic":
            h = ctypes.c_void_p()
            pw, dw, kw = _host_or_device(W, np.float64)
            _check(lib().qg_create_model_diabatic_rep(grid.handle, self.S, _dbl_array(self.mass), pw, dw,
                                                      ctypes.byref(h)), "qg_create_model_diabatic_rep")
            self.handle = h
        elif W is not None:
            self.handle = qg_create_model_diabatic(grid.handle, self.S, self.mass, W, dW)
        else:
            self.handle = qg_create_model(grid.handle, self.S, self.mass, V, F)

    def _rotate(self, psi, fn):
        shape = (self.S,) + tuple(self.grid.N)
        p, dev, keep = _host_or_device(psi, np.complex128)
        if dev:
            out = psi.new_empty(psi.shape)
        else:
            out = np.empty(shape, dtype=np.complex128)
        q, dq_, kq = _host_or_device(out, np.complex128)
        _check(getattr(lib(), fn)(self.handle, p, q, dev), fn)
        return out

    def to_adiabatic(self, psi_diab):
        """psi = O(q)^T psi_diab (Eq. psi_diab2adiab); models built from W."""
        return self._rotate(psi_diab, "qg_diabatic_to_adiabatic")

    def to_diabatic(self, psi_adiab):
        return self._rotate(psi_adiab, "qg_adiabatic_to_diabatic")

    def fields(self):
        g = self.grid
        V = np.empty((self.S,) + tuple(g.N))
        F = np.empty((g.D, self.S * (self.S - 1) // 2) + tuple(g.N))
        _check(lib().qg_model_fields(self.handle, ctypes.c_void_p(V.ctypes.data), ctypes.c_void_p(F.ctypes.data), 0),
               "qg_model_fields")
        return V, F

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qg_destroy_model(self.handle)
            self.handle = None


class State:
    def __init__(self, model, precision=QG_C128, stream=None):
        self.model = model
        self.shape = (model.S,) + tuple(model.grid.N)
        self.handle = qg_create_state(model.handle, precision)
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        _check(lib().qg_state_set_stream(self.handle, ctypes.c_void_p(raw or 0)), "qg_state_set_stream")

    def set(self, psi):
        p, dev, keep = _host_or_device(psi, np.complex128)
        _check(lib().qg_set_state(self.handle, p, dev), "qg_set_state")

    def get(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.complex128)
        p, dev, keep = _host_or_device(out, np.complex128)
        _check(lib().qg_get_state(self.handle, p, dev), "qg_get_state")
        return out

    def set_gaussian(self, surface, q0, p0, sigma0):
        _check(lib().qg_set_gaussian(self.handle, surface, _dbl_array(q0), _dbl_array(p0), _dbl_array(sigma0)),
               "qg_set_gaussian")

    def apply_h(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.complex128)
        p, dev, keep = _host_or_device(out, np.complex128)
        _check(lib().qg_apply_h(self.handle, p, dev), "qg_apply_h")
        return out

    def propagate(self, method, order, scheme, dt, nsteps, opts=None, allow_fail=False):
        st = StepStats()
        o = opts if opts is not None else default_solver_opts()
        r = lib().qg_propagate(self.handle, method, order, scheme, float(dt), int(nsteps), ctypes.byref(o),
                               ctypes.byref(st))
        _check(r, "qg_propagate", allow=(QG_ERR_NOT_CONVERGED,) if allow_fail else ())
        return st.as_dict()

    def step_implicit(self, method, order, scheme, dt, opts=None, allow_fail=False):
        st = StepStats()
        o = opts if opts is not None else default_solver_opts()
        r = lib().qg_step_implicit(self.handle, method, order, scheme, float(dt), ctypes.byref(o), ctypes.byref(st))
        _check(r, "qg_step_implicit", allow=(QG_ERR_NOT_CONVERGED,) if allow_fail else ())
        return st.as_dict()

    def set_launch_width(self, ctas):
        """2-D states: CTAs of the cooperative launch (0 = automatic)."""
        _check(lib().qg_state_set_launch_width(self.handle, int(ctas)), "qg_state_set_launch_width")

    def interpolate_from(self, other):
        """This state becomes the trigonometric interpolant of other's state
        on this state's grid (Appendix B)."""
        _check(lib().qg_interpolate(other.handle, self.handle), "qg_interpolate")

    def set_cluster(self, G):
        """1-D states: G = 0 one CTA with vectors in global memory; G = 1, 2,
        4, 8, 16 the shared-memory cluster form with G CTAs per instance."""
        _check(lib().qg_state_set_cluster(self.handle, int(G)), "qg_state_set_cluster")

    def autotune(self, method, order, scheme, dt, trial_steps=1, opts=None):
        """2-D states: pick the fastest cooperative launch width; returns the
        trial times (ms) at the automatic width, 1/2 and 1/4 of it."""
        o = opts if opts is not None else default_solver_opts()
        ms = (ctypes.c_double * 3)()
        _check(lib().qg_state_autotune(self.handle, method, order, scheme, float(dt), int(trial_steps),
                                       ctypes.byref(o), ms), "qg_state_autotune")
        return list(ms)

    def norm(self):
        v = ctypes.c_double()
        _check(lib().qg_norm(self.handle, ctypes.byref(v)), "qg_norm")
        return v.value

    def energy(self):
        v = ctypes.c_double()
        _check(lib().qg_energy(self.handle, ctypes.byref(v)), "qg_energy")
        return v.value

    def population(self):
        v = (ctypes.c_double * self.model.S)()
        _check(lib().qg_population(self.handle, v), "qg_population")
        return np.array(list(v))

    def overlap(self, other):
        v = (ctypes.c_double * 2)()
        _check(lib().qg_overlap(self.handle, other.handle, v), "qg_overlap")
        return complex(v[0], v[1])

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qg_destroy_state(self.handle)
            self.handle = None


def qg_batch_propagate(states, method, order, scheme, dt, nsteps, opts=None, allow_fail=False):
    """One persistent launch over all states; returns (statuses, per-state stats dicts)."""
    n = len(states)
    arr = (ctypes.c_void_p * n)(*[s.handle.value for s in states])
    stt = (ctypes.c_int32 * n)()
    sts = (StepStats * n)()
    o = opts if opts is not None else default_solver_opts()
    r = lib().qg_batch_propagate(arr, n, method, order, scheme, float(dt), int(nsteps), ctypes.byref(o), stt, sts)
    _check(r, "qg_batch_propagate", allow=(QG_ERR_NOT_CONVERGED,) if allow_fail else ())
    return list(stt), [s.as_dict() for s in sts]


class Batch:
    """Reusable batch of states for repeated one-launch propagation."""

    def __init__(self, states):
        self.states = list(states)
        n = len(self.states)
        arr = (ctypes.c_void_p * n)(*[s.handle.value for s in self.states])
        h = ctypes.c_void_p()
        _check(lib().qg_batch_create(arr, n, ctypes.byref(h)), "qg_batch_create")
        self.handle = h
        self._stt = (ctypes.c_int32 * n)()
        self._sts = (StepStats * n)()

    def run(self, method, order, scheme, dt, nsteps, opts=None, allow_fail=False, want_stats=True):
        o = opts if opts is not None else default_solver_opts()
        r = lib().qg_batch_run(self.handle, method, order, scheme, float(dt), int(nsteps), ctypes.byref(o),
                               self._stt, self._sts)
        _check(r, "qg_batch_run", allow=(QG_ERR_NOT_CONVERGED,) if allow_fail else ())
        if not want_stats:
            return None
        return list(self._stt), [s.as_dict() for s in self._sts]

    def capture(self, method, order, scheme, dt, nsteps, opts=None):
        o = opts if opts is not None else default_solver_opts()
        _check(lib().qg_batch_capture(self.handle, method, order, scheme, float(dt), int(nsteps), ctypes.byref(o)),
               "qg_batch_capture")

    def replay(self):
        _check(lib().qg_batch_replay(self.handle), "qg_batch_replay")

    def stats(self, allow_fail=False):
        r = lib().qg_batch_stats(self.handle, self._stt, self._sts)
        _check(r, "qg_batch_stats", allow=(QG_ERR_NOT_CONVERGED,) if allow_fail else ())
        return list(self._stt), [s.as_dict() for s in self._sts]

    def autotune(self, method, order, scheme, dt, trial_steps=1, opts=None):
        """Pick the fastest launch shape on the real batch; returns the trial
        times (ms) of {1, 2} CTAs/SM x {all surfaces, one surface} per FFT,
        then of the shared-memory cluster form at the smallest cluster size
        and at twice it (-1: does not fit)."""
        o = opts if opts is not None else default_solver_opts()
        ms = (ctypes.c_double * 6)()
        _check(lib().qg_batch_autotune(self.handle, method, order, scheme, float(dt), int(trial_steps),
                                       ctypes.byref(o), ms), "qg_batch_autotune")
        c, s = ctypes.c_int(), ctypes.c_int()
        _check(lib().qg_batch_tuning(self.handle, ctypes.byref(c), ctypes.byref(s)), "qg_batch_tuning")
        return {"trial_ms": list(ms), "ctas_per_sm": c.value, "surfaces_per_fft": s.value, "cluster": self.cluster,
                "classes": self.classes()}

    def classes(self):
        """Grid-size classes of the batch with their launch shapes."""
        nc = ctypes.c_int()
        arr = [(ctypes.c_int * 12)() for _ in range(5)]
        _check(lib().qg_batch_classes(self.handle, ctypes.byref(nc), *arr), "qg_batch_classes")
        keys = ["N", "count", "ctas_per_sm", "surfaces_per_fft", "cluster"]
        return [{k: a[c] for k, a in zip(keys, arr)} for c in range(nc.value)]

    @property
    def cluster(self):
        """Cluster size of the shared-memory cluster form (0: one-CTA form)."""
        g = ctypes.c_int()
        _check(lib().qg_batch_cluster(self.handle, ctypes.byref(g)), "qg_batch_cluster")
        return g.value

    def set_cluster(self, G):
        _check(lib().qg_batch_set_cluster(self.handle, int(G)), "qg_batch_set_cluster")

    @property
    def stream(self):
        return lib().qg_batch_stream(self.handle)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qg_batch_destroy(self.handle)
            self.handle = None


def cluster_size(N, S, restart=30):
    """Smallest cluster size of the shared-memory cluster form that holds an
    instance of N points and S surfaces (0: none)."""
    return int(lib().qg_cluster_size(int(N), int(S), int(restart)))


def probe_fp64():
    """Measured FP64 rates of the current device: FMA and add TFLOP/s, the
    instructions per SM per clock of each, and the SM clock (GHz) seen."""
    v = [ctypes.c_double() for _ in range(5)]
    _check(lib().qg_probe_fp64(*[ctypes.byref(x) for x in v]), "qg_probe_fp64")
    return dict(zip(["fma_tflops", "add_tflops", "fma_per_sm_clk", "add_per_sm_clk", "sm_ghz"], [x.value for x in v]))


def qg_version():
    return lib().qg_version().decode()
