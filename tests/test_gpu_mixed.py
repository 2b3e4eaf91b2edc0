"""Mixed-precision form: complex64 inner GMRES with FP64 residual refinement
(the state, the composition, the residual and the observables stay FP64).
Checked against the dense FP64 oracle and against the FP64 GPU path; the
error against the oracle is stated per case."""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import FS, nai_library_model, nai_oracle_fields, rel_l2
from oracle import grid as ogrid, hamiltonian as oham, initial as oinit, propagate as oprop

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method,order,scheme", [(0, 2, 0), (1, 4, 1), (1, 6, 0), (0, 8, 1)])
def test_mixed_vs_oracle_small(qglib, cuda, method, order, scheme):
    qmin, qmax, n = 3.8, 12.0, 128
    grid, model = nai_library_model(qglib, n, qmin, qmax)
    V, F = nai_oracle_fields(n, qmin, qmax)
    H = oham.dense_h([qmin], [qmax], [n], [wl.NAI_REDUCED_MASS], V, F)
    q, dq = ogrid.points(qmin, qmax, n)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [5.2], [4.0], [0.35]))
    st = qglib.State(model, precision=qglib.QG_C64_MIXED)
    st.set(psi0)
    opts = qglib.default_solver_opts(tol=1e-14)
    s = st.propagate(method, order, scheme, 1.0 * FS, 2, opts)
    want = oprop.DenseStepper(H).propagate(psi0, 1.0 * FS, 2, method, order, scheme)
    err = rel_l2(st.get(), want)
    print("mixed vs oracle (method %d order %d scheme %d): rel L2 %.2e, fp64 H psi %d, c64 H psi %d, outer %d" %
          (method, order, scheme, err, s["n_hpsi"], s["n_hpsi32"], s["n_outer"]))
    assert err < 1e-11
    assert s["n_hpsi32"] > 0 and s["n_outer"] >= s["n_substeps"]


def test_mixed_nai_like_n1024_trapezoidal_200_steps(qglib, cuda):
    n = 1024
    grid, model = nai_library_model(qglib, n)
    V, F = nai_oracle_fields(n)
    H = oham.dense_h([wl.NAI_QMIN], [wl.NAI_QMAX], [n], [wl.NAI_REDUCED_MASS], V, F)
    q, dq = ogrid.points(wl.NAI_QMIN, wl.NAI_QMAX, n)
    q0, p0, s0 = wl.initial_gaussian_params(0)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [q0], [p0], [s0]))
    want = oprop.DenseStepper(H).propagate(psi0, 0.1 * FS, 200, oprop.TRAPEZOIDAL, 2, 1)
    st = qglib.State(model, precision=qglib.QG_C64_MIXED)
    st.set_gaussian(1, [q0], [p0], [s0])
    st.propagate(qglib.QG_TRAPEZOIDAL, 2, qglib.QG_SUZUKI, 0.1 * FS, 200, qglib.default_solver_opts(tol=1e-14))
    err = rel_l2(st.get(), want)
    print("mixed N=1024 trapezoidal 200 steps: rel L2 vs oracle %.2e" % err)
    assert err < 1e-11


def test_mixed_equals_fp64_path_full_size(qglib, cuda):
    n = 2048
    grid, model = nai_library_model(qglib, n)
    a = qglib.State(model)
    b = qglib.State(model, precision=qglib.QG_C64_MIXED)
    for s in (a, b):
        s.set_gaussian(1, [wl.NAI_Q0], [wl.NAI_P0], [wl.NAI_SIGMA0])
    opts = qglib.default_solver_opts(tol=1e-13)
    sa = a.propagate(qglib.QG_MIDPOINT, 6, qglib.QG_SUZUKI, 0.5 * FS, 4, opts)
    sb = b.propagate(qglib.QG_MIDPOINT, 6, qglib.QG_SUZUKI, 0.5 * FS, 4, opts)
    err = rel_l2(b.get(), a.get())
    print("mixed vs fp64 path N=2048 Suzuki-6: rel L2 %.2e; fp64 H psi %d vs %d (+%d c64)" %
          (err, sa["n_hpsi"], sb["n_hpsi"], sb["n_hpsi32"]))
    assert err < 1e-11
    assert sb["n_hpsi"] < sa["n_hpsi"]
    assert abs(b.norm() - 1.0) < 1e-12


def test_mixed_not_converged_restores(qglib, cuda):
    qmin, qmax, n = 3.8, 12.0, 128
    grid, model = nai_library_model(qglib, n, qmin, qmax)
    st = qglib.State(model, precision=qglib.QG_C64_MIXED)
    st.set_gaussian(1, [5.0], [0.0], [0.4])
    before = st.get()
    opts = qglib.default_solver_opts(tol=1e-14, max_outer=1, max_iters=2, restart=2)
    s = st.propagate(qglib.QG_TRAPEZOIDAL, 2, 0, 3000.0 * FS, 2, opts, allow_fail=True)
    assert s["status"] == qglib.QG_ERR_NOT_CONVERGED
    np.testing.assert_array_equal(st.get(), before)


def test_mixed_order2_midpoint_hpsi_counts(qglib, cuda):
    # with a single fraction per step the mixed form starts each solve from a
    # complex64 explicit-Euler step and forms every FP64 residual exactly: one
    # FP64 H psi per refinement step plus the final check, one complex64 H psi
    # for the start plus one per inner iteration or inner restart
    n = 512
    grid, model = nai_library_model(qglib, n)
    st = qglib.State(model, precision=qglib.QG_C64_MIXED)
    st.set_gaussian(1, [wl.NAI_Q0], [1.0], [wl.NAI_SIGMA0])
    s = st.propagate(qglib.QG_MIDPOINT, 2, qglib.QG_SUZUKI, 0.5 * FS, 20, qglib.default_solver_opts(tol=1e-13))
    assert s["n_substeps"] == 20
    assert s["n_hpsi"] == s["n_outer"] + s["n_substeps"]
    assert s["n_hpsi32"] == s["n_substeps"] + s["n_krylov"] + s["n_restart"]
