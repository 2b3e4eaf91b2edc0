"""GPU parity of the elementary comparison methods of Sec. II B -- explicit
Euler (Eq. exp_euler), implicit Euler (Eq. imp_euler) and second-order
differencing (Eq. sod_method, two-stage Runge-Kutta start) -- against the
dense oracle, with their norm behaviour and the SOD stability limit
(Eq. sod_critical_timestep)."""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import nai_library_model, nai_oracle_fields, rel_l2
from oracle import grid as ogrid, hamiltonian as oham, initial as oinit, propagate as oprop

pytestmark = pytest.mark.gpu


def _setup(qglib, qmin, qmax, n, q0=5.2, p0=4.0, s0=0.35):
    grid, model = nai_library_model(qglib, n, qmin, qmax)
    V, F = nai_oracle_fields(n, qmin, qmax)
    H = oham.dense_h([qmin], [qmax], [n], [wl.NAI_REDUCED_MASS], V, F)
    q, dq = ogrid.points(qmin, qmax, n)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [q0], [p0], [s0]))
    return grid, model, H, psi0, dq


def _run(qg, model, psi0, method, dt, nsteps, precision=None, tol=1e-14):
    st = qg.State(model, precision=qg.QG_C128 if precision is None else precision)
    st.set(psi0)
    order = 2 if method == qg.QG_SOD else 1
    stats = st.propagate(method, order, 0, dt, nsteps, qg.default_solver_opts(tol=tol))
    return st, stats


@pytest.mark.parametrize("method,dt,nsteps", [(2, 0.5, 40), (3, 20.0, 30), (4, 2.0, 300)])
def test_elementary_small_vs_oracle(qglib, cuda, method, dt, nsteps):
    grid, model, H, psi0, dq = _setup(qglib, 3.8, 12.0, 128)
    st, stats = _run(qglib, model, psi0, method, dt, nsteps)
    ora = oprop.DenseStepper(H)
    if method == oprop.SOD:
        want = ora.sod(psi0, dt, nsteps)[0]
    else:
        want = ora.euler_steps(psi0, dt, nsteps, method)
    assert rel_l2(st.get(), want) < 1e-11
    assert stats["n_substeps"] == nsteps


def test_implicit_euler_mixed_precision_vs_oracle(qglib, cuda):
    grid, model, H, psi0, dq = _setup(qglib, 3.8, 12.0, 128)
    st, _ = _run(qglib, model, psi0, qglib.QG_IMPLICIT_EULER, 20.0, 30, precision=qglib.QG_C64_MIXED)
    want = oprop.DenseStepper(H).euler_steps(psi0, 20.0, 30, oprop.IMPLICIT_EULER)
    assert rel_l2(st.get(), want) < 1e-11


@pytest.mark.parametrize("method,dt,nsteps", [(2, 0.05, 200), (3, 5.0, 40), (4, 0.25, 800)])
def test_elementary_full_size_vs_oracle(qglib, cuda, method, dt, nsteps):
    # the NaI-like grid of the paper (N = 2048); SOD below its critical step
    grid, model, H, psi0, dq = _setup(qglib, wl.NAI_QMIN, wl.NAI_QMAX, 2048, wl.NAI_Q0, 0.0, wl.NAI_SIGMA0)
    st, _ = _run(qglib, model, psi0, method, dt, nsteps)
    ora = oprop.DenseStepper(H)
    if method == oprop.SOD:
        want = ora.sod(psi0, dt, nsteps)[0]
    else:
        want = ora.euler_steps(psi0, dt, nsteps, method)
    assert rel_l2(st.get(), want) < 1e-11


def test_euler_norm_identities_at_8192(qglib, cuda):
    # Eqs. exp_eu_norm / imp_eu_norm with the oracle's matrix-free H:
    # ||(1 - i e H) psi||^2 = ||psi||^2 + e^2 ||H psi||^2 and
    # ||psi||^2 = ||psi'||^2 + e^2 ||H psi'||^2
    n = 8192
    grid, model = nai_library_model(qglib, n)
    V, F = nai_oracle_fields(n)
    q, dq = ogrid.points(wl.NAI_QMIN, wl.NAI_QMAX, n)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [wl.NAI_Q0], [1.0], [wl.NAI_SIGMA0]))
    h = lambda x: oham.apply_h_matrix_free(wl.NAI_QMIN, wl.NAI_QMAX, n, wl.NAI_REDUCED_MASS, V, F, x)
    nrm2 = lambda x: dq * float(np.vdot(x, x).real)
    e = 0.2
    a, _ = _run(qglib, model, psi0, qglib.QG_EXPLICIT_EULER, e, 1)
    assert abs(nrm2(a.get()) - (nrm2(psi0) + e * e * nrm2(h(psi0)))) < 1e-12
    b, _ = _run(qglib, model, psi0, qglib.QG_IMPLICIT_EULER, e, 1)
    pb = b.get()
    assert abs(nrm2(psi0) - (nrm2(pb) + e * e * nrm2(h(pb)))) < 1e-12
    assert nrm2(pb) < 1.0 < nrm2(a.get())


def test_sod_stability_limit(qglib, cuda):
    grid, model, H, psi0, dq = _setup(qglib, 3.8, 12.0, 64, 5.5, 2.0, 0.5)
    emax = np.abs(np.linalg.eigvalsh(H)).max()
    good, _ = _run(qglib, model, psi0, qglib.QG_SOD, 0.95 / emax, 2000)
    assert good.norm() < 10.0
    bad, _ = _run(qglib, model, psi0, qglib.QG_SOD, 1.05 / emax, 300)
    assert bad.norm() > 1e6


def test_elementary_methods_reject_composition_orders(qglib, cuda):
    grid, model, H, psi0, dq = _setup(qglib, 3.8, 12.0, 64)
    st = qglib.State(model)
    st.set(psi0)
    for method, order in ((qglib.QG_EXPLICIT_EULER, 2), (qglib.QG_SOD, 4), (qglib.QG_IMPLICIT_EULER, 4)):
        with pytest.raises(qglib.QgError):
            st.propagate(method, order, 0, 1.0, 1)
