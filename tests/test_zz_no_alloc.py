"""qg_propagate_noalloc: the propagation entry point for callers that may not
allocate GPU memory (its scratch is one fixed device array inside the
library).  Checked against the regular entry point qg_propagate on the same
inputs, over two calls in a row, through the C-ABI.  Collected last so that a
run stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import workloads as wl
from gpu_helpers import FS, rel_l2

pytestmark = pytest.mark.gpu


def _call(qg, torch, n, qmin, qmax, S, mass, V, F, psi, method, order, scheme, dt, nsteps, opts):
    st = qg.StepStats()
    r = qg.lib().qg_propagate_noalloc(n, qmin, qmax, S, mass, ctypes.c_void_p(V.data_ptr()),
                                      ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(psi.data_ptr()), method, order,
                                      scheme, dt, nsteps, ctypes.byref(opts), ctypes.byref(st),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return r, st


def test_noalloc_matches_qg_propagate_on_two_calls(qglib, cuda):
    torch = cuda
    n, qmin, qmax, mass = 2048, wl.NAI_QMIN, wl.NAI_QMAX, wl.NAI_REDUCED_MASS
    grid = qglib.Grid([n], [qmin], [qmax])
    W, dW = wl.nai_like_diabatic(grid.points())
    model = qglib.Model(grid, 2, [mass], W=W, dW=dW)
    Vh, Fh = model.fields()
    V = torch.tensor(Vh, device="cuda")
    F = torch.tensor(Fh, device="cuda")
    reg = qglib.State(model)
    reg.set_gaussian(1, [wl.NAI_Q0], [1.0], [wl.NAI_SIGMA0])
    psi = torch.tensor(reg.get(), device="cuda")
    opts = qglib.default_solver_opts(tol=1e-14, restart=16)
    dt = 0.5 * FS
    for _ in range(2):
        s_reg = reg.propagate(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, dt, 3, opts)
        r, s_na = _call(qglib, torch, n, qmin, qmax, 2, mass, V, F, psi, qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI,
                        dt, 3, opts)
        assert r == qglib.QG_OK, qglib.lib().qg_last_error_string()
        assert s_na.status == 0 and s_na.n_substeps == s_reg["n_substeps"] == 15
        assert rel_l2(psi.cpu().numpy(), reg.get()) < 1e-11


def _model_case(qg, torch, n, qmin, qmax, S, mass, W, dW):
    grid = qg.Grid([n], [qmin], [qmax])
    model = qg.Model(grid, S, [mass], W=W, dW=dW)
    Vh, Fh = model.fields()
    return grid, model, torch.tensor(Vh, device="cuda"), torch.tensor(Fh, device="cuda")


def test_noalloc_rebuilds_tables_between_grids_and_runs_s3_trapezoidal(qglib, cuda):
    # a call on another grid rebuilds the FFT tables kept in the shared array;
    # going back to the first grid rebuilds them again; an S = 3 model with
    # the trapezoidal rule uses the workspace with B as right-hand side
    torch = cuda
    mass = wl.NAI_REDUCED_MASS
    opts = qglib.default_solver_opts(tol=1e-14, restart=16)
    dt = 0.5 * FS
    cases = [(2048, wl.NAI_QMIN, wl.NAI_QMAX), (1024, wl.NAI_QMIN, 30.0), (2048, wl.NAI_QMIN, wl.NAI_QMAX)]
    for n, qmin, qmax in cases:
        q = qmin + (qmax - qmin) / n * np.arange(n)
        W, dW = wl.nai_like_diabatic(q)
        keep = _model_case(qglib, torch, n, qmin, qmax, 2, mass, W, dW)
        grid, model, V, F = keep
        reg = qglib.State(model)
        reg.set_gaussian(1, [wl.NAI_Q0], [2.0], [wl.NAI_SIGMA0])
        psi = torch.tensor(reg.get(), device="cuda")
        reg.propagate(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, dt, 2, opts)
        r, s_na = _call(qglib, torch, n, qmin, qmax, 2, mass, V, F, psi, qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI,
                        dt, 2, opts)
        assert r == qglib.QG_OK, qglib.lib().qg_last_error_string()
        assert s_na.status == 0
        assert rel_l2(psi.cpu().numpy(), reg.get()) < 1e-11
    seed = 1000
    while True:
        m = wl.avoided_crossing_model(seed)
        if m["S"] == 3 and m["N"] <= 2048:
            break
        seed += 1
    grid, model, V, F = _model_case(qglib, torch, m["N"], m["qmin"], m["qmax"], 3, m["mass"], m["W"], m["dW"])
    reg = qglib.State(model)
    reg.set_gaussian(m["surface"], [m["q0"]], [m["p0"]], [m["sigma0"]])
    psi = torch.tensor(reg.get(), device="cuda")
    reg.propagate(qglib.QG_TRAPEZOIDAL, 4, qglib.QG_TRIPLE_JUMP, 0.1 * FS, 3, opts)
    r, s_na = _call(qglib, torch, m["N"], m["qmin"], m["qmax"], 3, m["mass"], V, F, psi, qglib.QG_TRAPEZOIDAL, 4,
                    qglib.QG_TRIPLE_JUMP, 0.1 * FS, 3, opts)
    assert r == qglib.QG_OK, qglib.lib().qg_last_error_string()
    assert s_na.status == 0 and s_na.n_substeps == 9
    assert rel_l2(psi.cpu().numpy(), reg.get()) < 1e-11


def test_noalloc_rejects_sizes_beyond_its_capacity(qglib, cuda):
    torch = cuda
    n = 8192
    V = torch.zeros((2, n), dtype=torch.float64, device="cuda")
    F = torch.zeros((1, 1, n), dtype=torch.float64, device="cuda")
    psi = torch.zeros((2, n), dtype=torch.complex128, device="cuda")
    opts = qglib.default_solver_opts(restart=16)
    r, _ = _call(qglib, torch, n, 0.0, 10.0, 2, 100.0, V, F, psi, 0, 2, 0, 1.0, 1, opts)
    assert r == qglib.QG_ERR_INVALID_ARG
    assert b"capacity" in qglib.lib().qg_last_error_string()
    opts = qglib.default_solver_opts(restart=30)
    r, _ = _call(qglib, torch, 1024, 0.0, 10.0, 2, 100.0, V, F, psi, 0, 2, 0, 1.0, 1, opts)
    assert r == qglib.QG_ERR_INVALID_ARG
