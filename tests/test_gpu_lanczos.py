"""Short-recurrence (Lanczos) minimal-residual solver for the implicit steps:
against the dense oracle, against the GMRES path, in the mixed-precision
form, and its H psi count."""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import FS, nai_library_model, nai_oracle_fields, rel_l2
from oracle import grid as ogrid, hamiltonian as oham, initial as oinit, propagate as oprop

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method,order,scheme,precision", [(0, 2, 0, 0), (1, 4, 1, 0), (1, 8, 0, 0), (1, 6, 1, 1)])
def test_lanczos_vs_oracle(qglib, cuda, method, order, scheme, precision):
    qmin, qmax, n = 3.8, 12.0, 128
    grid, model = nai_library_model(qglib, n, qmin, qmax)
    V, F = nai_oracle_fields(n, qmin, qmax)
    H = oham.dense_h([qmin], [qmax], [n], [wl.NAI_REDUCED_MASS], V, F)
    q, dq = ogrid.points(qmin, qmax, n)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [5.2], [4.0], [0.35]))
    st = qglib.State(model, precision=precision)
    st.set(psi0)
    opts = qglib.default_solver_opts(tol=1e-14, solver=qglib.QG_SOLVER_LANCZOS, true_residual=1)
    s = st.propagate(method, order, scheme, 1.0 * FS, 2, opts)
    want = oprop.DenseStepper(H).propagate(psi0, 1.0 * FS, 2, method, order, scheme)
    err = rel_l2(st.get(), want)
    print("lanczos vs oracle (method %d order %d scheme %d precision %d): %.2e, krylov/substep %.1f" %
          (method, order, scheme, precision, err, s["n_krylov"] / s["n_substeps"]))
    assert err < 1e-11


def test_lanczos_equals_gmres_full_size(qglib, cuda):
    n = 2048
    grid, model = nai_library_model(qglib, n)
    a, b = qglib.State(model), qglib.State(model)
    for s in (a, b):
        s.set_gaussian(1, [wl.NAI_Q0], [wl.NAI_P0], [wl.NAI_SIGMA0])
    ga = a.propagate(1, 6, 1, 0.5 * FS, 3, qglib.default_solver_opts(tol=1e-13))
    lb = b.propagate(1, 6, 1, 0.5 * FS, 3, qglib.default_solver_opts(tol=1e-13, solver=qglib.QG_SOLVER_LANCZOS))
    err = rel_l2(b.get(), a.get())
    print("lanczos vs gmres N=2048 Suzuki-6: %.2e; krylov/substep %.2f vs %.2f" %
          (err, lb["n_krylov"] / lb["n_substeps"], ga["n_krylov"] / ga["n_substeps"]))
    assert err < 1e-11
    # one exact H psi per composed step (3), then 1 + I per sub-step
    assert lb["n_hpsi"] == 3 + lb["n_substeps"] + lb["n_krylov"] + lb["n_restart"]


@pytest.mark.parametrize("restart,true_residual", [(4, 0), (5, 1)])
def test_lanczos_short_cycles_vs_oracle(qglib, cuda, restart, true_residual):
    """Cycles of four or five Lanczos columns (the shortest the library
    accepts for this solver): the FP64 solve forms its iterate X += V y at the
    end of every cycle and restarts from the true residual (Sec. II B's Krylov
    solve, restarted); the result must not depend on it."""
    qmin, qmax, n = 3.8, 12.0, 128
    grid, model = nai_library_model(qglib, n, qmin, qmax)
    V, F = nai_oracle_fields(n, qmin, qmax)
    H = oham.dense_h([qmin], [qmax], [n], [wl.NAI_REDUCED_MASS], V, F)
    q, dq = ogrid.points(qmin, qmax, n)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [5.2], [4.0], [0.35]))
    st = qglib.State(model)
    st.set(psi0)
    opts = qglib.default_solver_opts(tol=1e-14, restart=restart, max_iters=400, solver=qglib.QG_SOLVER_LANCZOS,
                                     true_residual=true_residual)
    s = st.propagate(1, 4, 1, 1.0 * FS, 2, opts)
    want = oprop.DenseStepper(H).propagate(psi0, 1.0 * FS, 2, 1, 4, 1)
    err = rel_l2(st.get(), want)
    print("lanczos restart %d: %.2e, restarts %d" % (restart, err, s["n_restart"]))
    assert s["n_restart"] > 0
    assert err < 1e-11


def test_lanczos_scale_safeguard_vs_oracle(qglib, cuda):
    """H scaled by 1e40 (V times 1e40, mass divided by 1e40) and dt divided by
    1e40 is the same evolution.  The Lanczos vectors grow by about |H| per
    column, so their tracked scales leave [1e-100, 1e100] within three columns
    and the solver's rescaling pass runs; the result must match the oracle."""
    lam = 1e40
    qmin, qmax, n = 3.8, 12.0, 128
    V, F = nai_oracle_fields(n, qmin, qmax)
    mass = wl.NAI_REDUCED_MASS / lam
    g = qglib.Grid([n], [qmin], [qmax])
    model = qglib.Model(g, 2, [mass], V=V * lam, F=F)
    H = oham.dense_h([qmin], [qmax], [n], [mass], V * lam, F)
    q, dq = ogrid.points(qmin, qmax, n)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [5.2], [4.0], [0.35]))
    st = qglib.State(model)
    st.set(psi0)
    opts = qglib.default_solver_opts(tol=1e-14, solver=qglib.QG_SOLVER_LANCZOS)
    dt = 1.0 * FS / lam
    s = st.propagate(1, 4, 1, dt, 2, opts)
    want = oprop.DenseStepper(H).propagate(psi0, dt, 2, 1, 4, 1)
    err = rel_l2(st.get(), want)
    print("lanczos with H x 1e40: %.2e, krylov/substep %.1f" % (err, s["n_krylov"] / s["n_substeps"]))
    assert s["n_krylov"] >= 3 * s["n_substeps"]
    assert err < 1e-11
