"""Oracle parity at the exact configuration the default benchmark times.

NaI-like model, N = 2048, S = 2, implicit midpoint (Eq. imp_midpoint)
composed by Suzuki's fractal to order 8 (Eq. suzukis_fractal), dt = 10500/1024
a.u., Lanczos minimal-residual solves started from the explicit-Euler step
built from the carried H psi, tol 1e-15, restart 30, several seeded packets in
one persistent batched launch with the autotuned launch shape, one launch per
composed step -- compared element by element with the dense oracle (LU per
distinct implicit step) over two composed steps (250 elementary steps).

Full-size members N = 4096 and 8192, whose shared-memory plan differs, are
checked inside a batch two ways: the NaI-like model through the implicit
equation of one midpoint step with the oracle's matrix-free H, and a
constant-coupling model through its closed form (for V = v0 1 and a constant
F_01 = c the eigen-channels of -i hbar F, (1, +-i)/sqrt2, evolve as
H = (hbar k +- hbar c)^2 / 2m + v0 per Fourier mode, so every composed step
multiplies each mode by prod_f R(f dt E), R(x) = (1 - i x/2)/(1 + i x/2)).
"""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import nai_library_model, nai_oracle_fields, rel_l2
from oracle import composition as ocomp, grid as ogrid, hamiltonian as oham, initial as oinit, propagate as oprop

pytestmark = pytest.mark.gpu

N_OP = 2048
DT_OP = 10500.0 / 1024
SEEDS = (0, 1, 2, 3)
STEPS = 2


def _op_opts(qg, **kw):
    base = dict(tol=1e-15, restart=30, max_iters=600, solver=qg.QG_SOLVER_LANCZOS, guess=qg.QG_GUESS_EULER)
    base.update(kw)
    return qg.default_solver_opts(**base)


@pytest.fixture(scope="module")
def op_reference():
    V, F = nai_oracle_fields(N_OP)
    H = oham.dense_h([wl.NAI_QMIN], [wl.NAI_QMAX], [N_OP], [wl.NAI_REDUCED_MASS], V, F)
    q, dq = ogrid.points(wl.NAI_QMIN, wl.NAI_QMAX, N_OP)
    psi0 = []
    for seed in SEEDS:
        q0, p0, s0 = wl.initial_gaussian_params(seed)
        psi0.append(oinit.state_on_surface(2, 1, oinit.gaussian([q], [q0], [p0], [s0])))
    st = oprop.DenseStepper(H)
    one = st.propagate_columns(psi0, DT_OP, 1, oprop.MIDPOINT, 8, ocomp.SUZUKI)
    two = st.propagate_columns(one, DT_OP, 1, oprop.MIDPOINT, 8, ocomp.SUZUKI)
    return dict(psi0=psi0, after=[one, two], dq=dq)


def _op_batch(qg, precision):
    grid, model = nai_library_model(qg, N_OP)
    states = []
    for seed in SEEDS:
        st = qg.State(model, precision=precision)
        q0, p0, s0 = wl.initial_gaussian_params(seed)
        st.set_gaussian(1, [q0], [p0], [s0])
        states.append(st)
    return grid, model, states


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_operating_point_batched_vs_oracle(qglib, cuda, op_reference, precision):
    qg = qglib
    prec = qg.QG_C64_MIXED if precision == "mixed" else qg.QG_C128
    grid, model, states = _op_batch(qg, prec)
    for st, want in zip(states, op_reference["psi0"]):
        assert rel_l2(st.get(), want) < 1e-13
    batch = qg.Batch(states)
    opts = _op_opts(qg)
    batch.autotune(qg.QG_MIDPOINT, 8, qg.QG_SUZUKI, DT_OP, 1, opts)   # restores the states
    for k in range(STEPS):
        stt, stats = batch.run(qg.QG_MIDPOINT, 8, qg.QG_SUZUKI, DT_OP, 1, opts)
        assert stt == [0] * len(SEEDS)
        for s in stats:
            assert s["n_substeps"] == 125
            # carried H psi: one exact H psi per composed step plus one per
            # Krylov iteration or residual
            assert s["n_hpsi"] >= 1
        for st, want in zip(states, op_reference["after"][k]):
            assert rel_l2(st.get(), want) < 1e-11
    for st in states:
        assert abs(st.norm() - 1.0) < 1e-12


def test_operating_point_single_state_equals_batch_member(qglib, cuda, op_reference):
    # the per-instance entry point at the same point agrees with the oracle too
    qg = qglib
    grid, model, states = _op_batch(qg, qg.QG_C128)
    st = states[0]
    st.propagate(qg.QG_MIDPOINT, 8, qg.QG_SUZUKI, DT_OP, STEPS, _op_opts(qg))
    assert rel_l2(st.get(), op_reference["after"][STEPS - 1][0]) < 1e-11


def _const_coupling_exact(psi0, qmin, qmax, n, m, v0, c, dt, nsteps, order, scheme):
    k = ogrid.wavenumbers(qmin, qmax, n)
    a, b = np.fft.fft(psi0[0]), np.fft.fft(psi0[1])
    plus, minus = (a - 1j * b) / np.sqrt(2), (a + 1j * b) / np.sqrt(2)
    for sign, amp in ((1.0, "plus"), (-1.0, "minus")):
        E = (k + sign * c) ** 2 / (2.0 * m) + v0
        g = np.ones(n, dtype=np.complex128)
        for f in ocomp.schedule(order, scheme):
            x = f * dt * E
            g *= (1 - 0.5j * x) / (1 + 0.5j * x)
        if amp == "plus":
            plus = plus * g ** nsteps
        else:
            minus = minus * g ** nsteps
    out0 = (plus + minus) / np.sqrt(2)
    out1 = 1j * (plus - minus) / np.sqrt(2)
    return np.stack([np.fft.ifft(out0), np.fft.ifft(out1)])


def test_full_size_members_closed_form_in_batch(qglib, cuda):
    # constant-coupling models at N = 2048, 4096, 8192 in one batch at the
    # operating point (Suzuki 8, dt = 10.25 a.u., Lanczos, tol 1e-15)
    qg = qglib
    qmin, qmax = wl.NAI_QMIN, wl.NAI_QMAX
    m, v0, c = wl.NAI_REDUCED_MASS, 0.01, 2.0
    keep, states, wants = [], [], []
    for n in (8192, 2048, 4096):
        g = qg.Grid([n], [qmin], [qmax])
        V = np.full((2, n), v0)
        F = np.full((1, 1, n), c)
        lm = qg.Model(g, 2, [m], V=V, F=F)
        q, dq = ogrid.points(qmin, qmax, n)
        psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [20.0], [6.0], [0.4]))
        st = qg.State(lm)
        st.set(psi0)
        keep += [g, lm]
        states.append(st)
        wants.append(_const_coupling_exact(psi0, qmin, qmax, n, m, v0, c, DT_OP, 2, 8, ocomp.SUZUKI))
    batch = qg.Batch(states)
    opts = _op_opts(qg)
    batch.autotune(qg.QG_MIDPOINT, 8, qg.QG_SUZUKI, DT_OP, 1, opts)
    stt, stats = batch.run(qg.QG_MIDPOINT, 8, qg.QG_SUZUKI, DT_OP, 2, opts)
    assert stt == [0, 0, 0]
    for st, want in zip(states, wants):
        assert rel_l2(st.get(), want) < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_nai_members_implicit_equation_in_batch(qglib, cuda, precision):
    # NaI-like members N = 2048, 4096, 8192 in one batch, one order-2 midpoint
    # step at dt = 10.25 a.u.: chi = (psi0 + psi1)/2 must solve
    # (1 + i tau H) chi = psi0 with the oracle's matrix-free H
    qg = qglib
    prec = qg.QG_C64_MIXED if precision == "mixed" else qg.QG_C128
    keep, states, psi0s, fields = [], [], [], []
    for n in (4096, 2048, 8192):
        grid, model = nai_library_model(qg, n)
        q, dq = ogrid.points(wl.NAI_QMIN, wl.NAI_QMAX, n)
        psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [wl.NAI_Q0], [3.0], [wl.NAI_SIGMA0]))
        st = qg.State(model, precision=prec)
        st.set(psi0)
        keep += [grid, model]
        states.append(st)
        psi0s.append(psi0)
        fields.append(nai_oracle_fields(n))
    batch = qg.Batch(states)
    stt, _ = batch.run(qg.QG_MIDPOINT, 2, qg.QG_SUZUKI, DT_OP, 1, _op_opts(qg))
    assert stt == [0, 0, 0]
    tau = DT_OP / 2
    for st, psi0, (V, F) in zip(states, psi0s, fields):
        n = psi0.shape[1]
        chi = 0.5 * (psi0 + st.get())
        Hchi = oham.apply_h_matrix_free(wl.NAI_QMIN, wl.NAI_QMAX, n, wl.NAI_REDUCED_MASS, V, F, chi)
        r = chi + 1j * tau * Hchi - psi0
        assert np.linalg.norm(r) / np.linalg.norm(psi0) < 1e-13


@pytest.mark.parametrize("G", [4, 8])
def test_operating_point_cluster_batch_vs_oracle(qglib, cuda, op_reference, G):
    # the same point in the shared-memory cluster form, one launch per step
    qg = qglib
    grid, model, states = _op_batch(qg, qg.QG_C128)
    batch = qg.Batch(states)
    batch.set_cluster(G)
    opts = _op_opts(qg)
    for k in range(STEPS):
        stt, stats = batch.run(qg.QG_MIDPOINT, 8, qg.QG_SUZUKI, DT_OP, 1, opts)
        assert stt == [0] * len(SEEDS)
        for st, want in zip(states, op_reference["after"][k]):
            assert rel_l2(st.get(), want) < 1e-11
