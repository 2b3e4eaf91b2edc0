"""The shared-memory cluster form of the 1-D propagator (one instance per
thread-block cluster, every solver vector in shared memory, the spectral
derivative split into per-CTA transforms and cross-CTA transforms through
distributed shared memory): parity with the dense oracle for every cluster
size, both Krylov solvers, both rules, S = 2 and 3, the elementary methods,
and equality with the one-CTA form."""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import FS, nai_library_model, nai_oracle_fields, rel_l2
from oracle import grid as ogrid, hamiltonian as oham, initial as oinit, propagate as oprop

pytestmark = pytest.mark.gpu

SMALL = (3.8, 12.0, 128)


@pytest.fixture(scope="module")
def small_case():
    qmin, qmax, n = SMALL
    V, F = nai_oracle_fields(n, qmin, qmax)
    H = oham.dense_h([qmin], [qmax], [n], [wl.NAI_REDUCED_MASS], V, F)
    q, dq = ogrid.points(qmin, qmax, n)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [5.2], [4.0], [0.35]))
    return H, psi0


def test_cluster_sizes_reported(qglib, cuda):
    assert qglib.cluster_size(2048, 2) == 4
    assert qglib.cluster_size(8192, 2) == 16
    assert qglib.cluster_size(512, 2) == 1
    assert qglib.cluster_size(8192, 3) == 0


@pytest.mark.parametrize("G", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("solver", [0, 1])
def test_cluster_small_vs_oracle(qglib, cuda, small_case, G, solver):
    H, psi0 = small_case
    qmin, qmax, n = SMALL
    grid, model = nai_library_model(qglib, n, qmin, qmax)
    st = qglib.State(model)
    st.set_cluster(G)
    st.set(psi0)
    opts = qglib.default_solver_opts(tol=1e-14, solver=solver)
    s = st.propagate(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, 1.0 * FS, 2, opts)
    want = oprop.DenseStepper(H).propagate(psi0, 1.0 * FS, 2, oprop.MIDPOINT, 4, 1)
    assert rel_l2(st.get(), want) < 1e-11
    assert s["n_substeps"] == 10 and s["status"] == 0


@pytest.mark.parametrize("method,order,scheme", [(0, 2, 1), (0, 6, 0), (1, 8, 2), (4, 2, 0), (3, 1, 0)])
def test_cluster_methods_vs_oracle(qglib, cuda, small_case, method, order, scheme):
    H, psi0 = small_case
    qmin, qmax, n = SMALL
    grid, model = nai_library_model(qglib, n, qmin, qmax)
    st = qglib.State(model)
    st.set_cluster(4)
    st.set(psi0)
    dt = 2.0 if method >= 2 else 1.0 * FS
    nsteps = 50 if method == oprop.SOD else 2
    st.propagate(method, order, scheme, dt, nsteps, qglib.default_solver_opts(tol=1e-14, solver=1))
    ora = oprop.DenseStepper(H)
    if method == oprop.SOD:
        want = ora.sod(psi0, dt, nsteps)[0]
    elif method == oprop.IMPLICIT_EULER:
        want = ora.euler_steps(psi0, dt, nsteps, method)
    else:
        want = ora.propagate(psi0, dt, nsteps, method, order, scheme)
    assert rel_l2(st.get(), want) < 1e-11


def test_cluster_three_surfaces_vs_oracle(qglib, cuda):
    from oracle import fields as ofields
    seed = 1000
    while True:
        m = wl.avoided_crossing_model(seed)
        if m["S"] == 3 and m["N"] <= 1024:
            break
        seed += 1
    g = qglib.Grid([m["N"]], [m["qmin"]], [m["qmax"]])
    lm = qglib.Model(g, 3, [m["mass"]], W=m["W"], dW=m["dW"])
    V, F, _ = ofields.general_adiabatic(m["W"], m["dW"], 3)
    q, dq = ogrid.points(m["qmin"], m["qmax"], m["N"])
    psi0 = oinit.state_on_surface(3, m["surface"], oinit.gaussian([q], [m["q0"]], [m["p0"]], [m["sigma0"]]))
    H = oham.dense_h([m["qmin"]], [m["qmax"]], [m["N"]], [m["mass"]], V, F)
    want = oprop.DenseStepper(H).propagate(psi0, 0.1 * FS, 2, oprop.MIDPOINT, 4, 1)
    G0 = qglib.cluster_size(m["N"], 3)
    assert G0 > 0
    for G in (G0, 2 * G0):
        st = qglib.State(lm)
        st.set_cluster(G)
        st.set(psi0)
        st.propagate(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, 0.1 * FS, 2, qglib.default_solver_opts(tol=1e-14))
        assert rel_l2(st.get(), want) < 1e-11


@pytest.mark.parametrize("n,G", [(1024, 2), (2048, 4), (2048, 8), (4096, 8), (8192, 16)])
def test_cluster_equals_one_cta_form_full_size(qglib, cuda, n, G):
    grid, model = nai_library_model(qglib, n)
    a, b = qglib.State(model), qglib.State(model)
    b.set_cluster(G)
    for st in (a, b):
        st.set_gaussian(1, [wl.NAI_Q0], [2.0], [wl.NAI_SIGMA0])
    opts = qglib.default_solver_opts(tol=1e-15, max_iters=600, solver=qglib.QG_SOLVER_LANCZOS)
    sa = a.propagate(qglib.QG_MIDPOINT, 8, qglib.QG_SUZUKI, 10500.0 / 1024, 1, opts)
    sb = b.propagate(qglib.QG_MIDPOINT, 8, qglib.QG_SUZUKI, 10500.0 / 1024, 1, opts)
    assert rel_l2(b.get(), a.get()) < 1e-12
    assert abs(sb["n_hpsi"] - sa["n_hpsi"]) <= 0.02 * sa["n_hpsi"]


def test_cluster_rejects_what_it_cannot_hold(qglib, cuda):
    grid, model = nai_library_model(qglib, 2048)
    st = qglib.State(model)
    with pytest.raises(qglib.QgError):
        st.set_cluster(2)          # 2 x 2048 / 2 values per CTA: too many
    mixed = qglib.State(model, precision=qglib.QG_C64_MIXED)
    with pytest.raises(qglib.QgError):
        mixed.set_cluster(4)
