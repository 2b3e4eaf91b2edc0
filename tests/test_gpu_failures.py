"""Failure detection without a GPU fault: bounded waits that run out return a
status, non-finite input makes the implicit solve fail and restores the
state, invalid handles and sizes are rejected on the host."""
import ctypes

import numpy as np
import pytest

import workloads as wl
from gpu_helpers import FS, nai_library_model

pytestmark = pytest.mark.gpu


def test_grid_barrier_wait_runs_out(qglib, cuda):
    t, p = ctypes.c_int(-1), ctypes.c_int(-1)
    r = qglib.lib().qg_selftest_barrier_timeout(ctypes.byref(t), ctypes.byref(p))
    assert r == qglib.QG_ERR_TIMEOUT and t.value == 1 and p.value == 0
    # the context is still usable afterwards
    grid, model = nai_library_model(qglib, 64, 3.8, 12.0)
    st = qglib.State(model)
    st.set_gaussian(1, [5.0], [0.0], [0.4])
    assert abs(st.norm() - 1.0) < 1e-13


def test_non_finite_state_fails_and_is_restored(qglib, cuda):
    grid, model = nai_library_model(qglib, 64, 3.8, 12.0)
    st = qglib.State(model)
    st.set_gaussian(1, [5.0], [0.0], [0.4])
    psi = st.get()
    psi[1, 10] = np.nan
    st.set(psi)
    s = st.propagate(0, 2, 0, 1.0 * FS, 2, qglib.default_solver_opts(max_iters=50), allow_fail=True)
    assert s["status"] == qglib.QG_ERR_NOT_CONVERGED
    after = st.get()
    assert np.isnan(after[1, 10]) and np.array_equal(after[~np.isnan(after)], psi[~np.isnan(psi)])


def test_invalid_calls_are_rejected_before_device_work(qglib, cuda):
    L = qglib.lib()
    assert L.qg_propagate(None, 0, 2, 0, 1.0, 1, None, None) == qglib.QG_ERR_INVALID_ARG
    assert L.qg_set_state(None, None, 0) == qglib.QG_ERR_INVALID_ARG
    grid, model = nai_library_model(qglib, 64, 3.8, 12.0)
    st = qglib.State(model)
    assert L.qg_set_gaussian(st.handle, 5, (ctypes.c_double * 1)(5.0), (ctypes.c_double * 1)(0.0),
                             (ctypes.c_double * 1)(0.4)) == qglib.QG_ERR_INVALID_ARG
    assert L.qg_set_gaussian(st.handle, 1, (ctypes.c_double * 1)(5.0), (ctypes.c_double * 1)(0.0),
                             (ctypes.c_double * 1)(-1.0)) == qglib.QG_ERR_INVALID_ARG
    assert L.qg_propagate_ex(st.handle, 2, 0, 2, 0, 1.0, 1, None, None) == qglib.QG_ERR_INVALID_ARG   # no buffers
    assert L.qg_create_state(model.handle, 7, ctypes.byref(ctypes.c_void_p())) == qglib.QG_ERR_INVALID_ARG
