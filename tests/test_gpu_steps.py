"""GPU parity of the composed implicit steps (Secs. II B-C) against the dense
CPU oracle, and the method's invariants measured on the GPU path."""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import FS, nai_library_model, nai_oracle_fields, rel_l2
from oracle import composition as ocomp, grid as ogrid, hamiltonian as oham, initial as oinit, \
    observables as oobs, propagate as oprop

pytestmark = pytest.mark.gpu

SMALL = (3.8, 12.0, 128)


def _small_setup(qglib):
    qmin, qmax, n = SMALL
    grid, model = nai_library_model(qglib, n, qmin, qmax)
    V, F = nai_oracle_fields(n, qmin, qmax)
    H = oham.dense_h([qmin], [qmax], [n], [wl.NAI_REDUCED_MASS], V, F)
    q, dq = ogrid.points(qmin, qmax, n)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [5.2], [4.0], [0.35]))
    return grid, model, H, psi0


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("order,scheme", [(2, 0), (4, 0), (4, 1), (6, 0), (6, 1), (8, 0), (8, 1), (6, 2), (8, 2)])
def test_composed_steps_vs_oracle(qglib, cuda, method, order, scheme):
    grid, model, H, psi0 = _small_setup(qglib)
    dt = 1.0 * FS
    st = qglib.State(model)
    st.set(psi0)
    opts = qglib.default_solver_opts(tol=1e-14)
    stats = st.propagate(method, order, scheme, dt, 2, opts)
    want = oprop.DenseStepper(H).propagate(psi0, dt, 2, method, order, scheme)
    assert rel_l2(st.get(), want) < 1e-11
    assert stats["n_substeps"] == 2 * len(ocomp.schedule(order, scheme))


def test_midpoint_epilogue_as_written_vs_oracle(qglib, cuda):
    grid, model, H, psi0 = _small_setup(qglib)
    st = qglib.State(model)
    st.set(psi0)
    opts = qglib.default_solver_opts(tol=1e-14, midpoint_epilogue=1)
    st.propagate(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, 2.0 * FS, 2, opts)
    want = oprop.DenseStepper(H).propagate(psi0, 2.0 * FS, 2, oprop.MIDPOINT, 4, 1)
    assert rel_l2(st.get(), want) < 1e-11


@pytest.mark.parametrize("seed", [0, 1])
def test_nai_like_n1024_trapezoidal_200_steps(qglib, cuda, seed):
    # N = 1024, trapezoidal rule, dt = 0.1 fs, 200 steps; Gaussian on the
    # excited surface with a seeded centre and width
    n = 1024
    grid, model = nai_library_model(qglib, n)
    V, F = nai_oracle_fields(n)
    H = oham.dense_h([wl.NAI_QMIN], [wl.NAI_QMAX], [n], [wl.NAI_REDUCED_MASS], V, F)
    q, dq = ogrid.points(wl.NAI_QMIN, wl.NAI_QMAX, n)
    q0, p0, s0 = wl.initial_gaussian_params(seed)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [q0], [p0], [s0]))
    want = oprop.DenseStepper(H).propagate(psi0, 0.1 * FS, 200, oprop.TRAPEZOIDAL, 2, 1)
    st = qglib.State(model)
    st.set_gaussian(1, [q0], [p0], [s0])
    assert rel_l2(st.get(), psi0) < 1e-13
    st.propagate(qglib.QG_TRAPEZOIDAL, 2, qglib.QG_SUZUKI, 0.1 * FS, 200, qglib.default_solver_opts(tol=1e-14))
    assert rel_l2(st.get(), want) < 1e-11
    # the production tolerance 1e-12: each implicit solve errs by at most
    # tol * ||b|| because ||(1 + i tau H)^{-1}|| <= 1
    st.set_gaussian(1, [q0], [p0], [s0])
    st.propagate(qglib.QG_TRAPEZOIDAL, 2, qglib.QG_SUZUKI, 0.1 * FS, 200, qglib.default_solver_opts(tol=1e-12))
    assert rel_l2(st.get(), want) < 200 * 1e-12


def test_nai_like_n2048_suzuki4_midpoint_vs_oracle(qglib, cuda):
    n = 2048
    grid, model = nai_library_model(qglib, n)
    V, F = nai_oracle_fields(n)
    H = oham.dense_h([wl.NAI_QMIN], [wl.NAI_QMAX], [n], [wl.NAI_REDUCED_MASS], V, F)
    q, dq = ogrid.points(wl.NAI_QMIN, wl.NAI_QMAX, n)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [wl.NAI_Q0], [0.0], [wl.NAI_SIGMA0]))
    want = oprop.DenseStepper(H).propagate(psi0, 1.0 * FS, 2, oprop.MIDPOINT, 4, 1)
    st = qglib.State(model)
    st.set(psi0)
    st.propagate(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, 1.0 * FS, 2, qglib.default_solver_opts(tol=1e-14))
    assert rel_l2(st.get(), want) < 1e-11


@pytest.mark.parametrize("n", [4096, 8192])
def test_full_size_implicit_solve_residual(qglib, cuda, n):
    # property at any size: after one trapezoidal step psi1 solves
    # (1 + i tau H) psi1 = (1 - i tau H) psi0, checked with the oracle's H
    grid, model = nai_library_model(qglib, n)
    V, F = nai_oracle_fields(n)
    q, dq = ogrid.points(wl.NAI_QMIN, wl.NAI_QMAX, n)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [wl.NAI_Q0], [2.0], [wl.NAI_SIGMA0]))
    dt = 0.5 * FS
    st = qglib.State(model)
    st.set(psi0)
    st.propagate(qglib.QG_TRAPEZOIDAL, 2, qglib.QG_SUZUKI, dt, 1, qglib.default_solver_opts(tol=1e-14))
    psi1 = st.get()
    tau = dt / 2
    h = lambda x: oham.apply_h_matrix_free(wl.NAI_QMIN, wl.NAI_QMAX, n, wl.NAI_REDUCED_MASS, V, F, x)
    b = psi0 - 1j * tau * h(psi0)
    r = psi1 + 1j * tau * h(psi1) - b
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-12


@pytest.mark.parametrize("order,steps", [(2, 400), (4, 100)])
def test_invariants_and_reversibility(qglib, cuda, order, steps):
    # Theorem (Sec. II C) and Fig. 6: norm, energy, symplectic form and time
    # reversibility conserved by the trapezoidal rule and its composition at
    # dt = 5 a.u. with the implicit steps solved to machine accuracy; the paper
    # reports residual errors below 2e-12
    n = 2048
    grid, model = nai_library_model(qglib, n)
    a, b = qglib.State(model), qglib.State(model)
    a.set_gaussian(1, [wl.NAI_Q0], [wl.NAI_P0], [wl.NAI_SIGMA0])
    b.set_gaussian(1, [wl.PHI_Q0], [wl.PHI_P0], [wl.NAI_SIGMA0])
    psi0 = a.get()
    n0, e0, w0 = a.norm(), a.energy(), -2 * a.overlap(b).imag
    opts = qglib.default_solver_opts(tol=1e-15, max_iters=2000)
    dt = 5.0
    a.propagate(qglib.QG_TRAPEZOIDAL, order, qglib.QG_SUZUKI, dt, steps, opts)
    b.propagate(qglib.QG_TRAPEZOIDAL, order, qglib.QG_SUZUKI, dt, steps, opts)
    assert abs(a.norm() - n0) < 2e-12
    assert abs(a.energy() - e0) < 2e-12
    assert abs(-2 * a.overlap(b).imag - w0) < 2e-12
    a.propagate(qglib.QG_TRAPEZOIDAL, order, qglib.QG_SUZUKI, -dt, steps, opts)
    dq = (wl.NAI_QMAX - wl.NAI_QMIN) / n
    assert np.linalg.norm(a.get() - psi0) * np.sqrt(dq) < 2e-12


def test_trapezoidal_equals_midpoint_on_gpu(qglib, cuda):
    n = 2048
    grid, model = nai_library_model(qglib, n)
    a, b = qglib.State(model), qglib.State(model)
    for s in (a, b):
        s.set_gaussian(1, [wl.NAI_Q0], [wl.NAI_P0], [wl.NAI_SIGMA0])
    opts = qglib.default_solver_opts(tol=1e-14)
    a.propagate(qglib.QG_TRAPEZOIDAL, 6, qglib.QG_SUZUKI, 2.0 * FS, 1, opts)
    b.propagate(qglib.QG_MIDPOINT, 6, qglib.QG_SUZUKI, 2.0 * FS, 1, opts)
    assert rel_l2(a.get(), b.get()) < 1e-11


@pytest.mark.parametrize("method,epi,extra,per_step", [(0, 0, 3, 0), (1, 1, 3, 0), (1, 0, 1, 1)])
def test_cost_model_counts(qglib, cuda, method, epi, extra, per_step):
    # Table I: (3 + I) H psi per elementary step.  With psi' = 2 chi - psi the
    # midpoint rule carries H psi from one sub-step to the next, so its
    # explicit-Euler start is free: 1 + I per sub-step, plus one exact H psi
    # per composed step.
    grid, model, H, psi0 = _small_setup(qglib)
    st = qglib.State(model)
    st.set(psi0)
    opts = qglib.default_solver_opts(tol=1e-13, restart=64, midpoint_epilogue=epi)
    s = st.propagate(method, 4, 0, 1.0 * FS, 2, opts)
    assert s["n_substeps"] == 6
    assert s["n_hpsi"] == extra * s["n_substeps"] + per_step * 2 + s["n_krylov"] + s["n_restart"]
    assert 0 < s["max_krylov"] <= opts.max_iters


def test_not_converged_restores_the_state(qglib, cuda):
    grid, model, H, psi0 = _small_setup(qglib)
    st = qglib.State(model)
    st.set(psi0)
    before = st.get()
    opts = qglib.default_solver_opts(tol=1e-14, max_iters=3, restart=3)
    s = st.propagate(qglib.QG_TRAPEZOIDAL, 2, 0, 2000.0 * FS, 3, opts, allow_fail=True)
    assert s["status"] == qglib.QG_ERR_NOT_CONVERGED
    assert s["failed_step"] == 0
    np.testing.assert_array_equal(st.get(), before)


def test_batch_equals_individual_launches(qglib, cuda):
    specs = [(256, 2, 1), (512, 3, 2), (64, 4, 3), (128, 2, 4)]
    states, refs = [], []
    keep = []
    for n, S, seed in specs:
        V, F = wl.random_adiabatic_fields(S, 1, (n,), seed=seed, v_scale=0.02, f_scale=0.3)
        psi = wl.random_psi(S, (n,), seed=seed + 10, smooth=n // 6)
        g = qglib.Grid([n], [-4.0], [4.0])
        m = qglib.Model(g, S, [30.0], V=V, F=F)
        a, b = qglib.State(m), qglib.State(m)
        a.set(psi)
        b.set(psi)
        keep += [g, m]
        states.append(a)
        refs.append(b)
    opts = qglib.default_solver_opts(tol=1e-13)
    stt, stats = qglib.qg_batch_propagate(states, qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, 0.05, 3, opts)
    assert stt == [0] * len(specs)
    for a, b in zip(states, refs):
        b.propagate(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, 0.05, 3, opts)
        np.testing.assert_array_equal(a.get(), b.get())


def test_invalid_arguments(qglib, cuda):
    with pytest.raises(qglib.QgError):
        qglib.Grid([100], [0.0], [1.0])          # not a power of two
    with pytest.raises(qglib.QgError):
        qglib.Grid([16384], [0.0], [1.0])        # above the maximum size
    with pytest.raises(qglib.QgError):
        qglib.Grid([64], [1.0], [1.0])           # empty interval
    grid, model, H, psi0 = _small_setup(qglib)
    st = qglib.State(model)
    for kw in (dict(order=3), dict(order=10), dict(scheme=7), dict(method=5)):
        a = dict(method=0, order=2, scheme=0)
        a.update(kw)
        with pytest.raises(qglib.QgError):
            st.propagate(a["method"], a["order"], a["scheme"], 1.0, 1)
    with pytest.raises(qglib.QgError):
        st.propagate(0, 2, 0, 1.0, 1, qglib.default_solver_opts(restart=65))
