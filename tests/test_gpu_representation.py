"""The diabatic representation (Sec. II E) and the changes of representation
and of grid (Eq. psi_diab2adiab, Appendix B) on the GPU, against the oracle."""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import FS, rel_l2
from oracle import fields as ofields, grid as ogrid, initial as oinit, propagate as oprop, representation as orep

pytestmark = pytest.mark.gpu


def _two_state(q):
    kf, a, d0 = 0.05, 0.6, 0.01
    c, w, c0 = 0.004, 1.0, 0.0015
    w11 = 0.5 * kf * (q - a) ** 2
    w22 = 0.5 * kf * (q + a) ** 2 + d0
    w12 = c * np.exp(-q ** 2 / (2 * w * w)) + c0
    d11 = kf * (q - a)
    d22 = kf * (q + a)
    d12 = -q / (w * w) * c * np.exp(-q ** 2 / (2 * w * w))
    return np.stack([w11, w12, w22]), np.stack([d11, d12, d22])[None]


def _three_state(q):
    A = np.random.default_rng(4).standard_normal((6, 3))
    W = np.stack([A[t, 0] + A[t, 1] * np.sin(q) + A[t, 2] * q * 0.1 for t in range(6)]) * 0.1
    dW = np.stack([A[t, 1] * np.cos(q) + A[t, 2] * 0.1 for t in range(6)])[None] * 0.1
    return W, dW


@pytest.mark.parametrize("method,order,scheme,solver,prec", [(1, 4, 1, 1, 0), (0, 6, 0, 0, 0), (1, 8, 2, 1, 0),
                                                             (1, 4, 1, 1, 1), (4, 2, 0, 1, 0)])
def test_diabatic_propagation_vs_oracle(qglib, cuda, method, order, scheme, solver, prec):
    qmin, qmax, n = 3.8, 12.0, 128
    q, dq = ogrid.points(qmin, qmax, n)
    W, dW = wl.nai_like_diabatic(q)
    g = qglib.Grid([n], [qmin], [qmax])
    m = qglib.Model(g, 2, [wl.NAI_REDUCED_MASS], W=W, representation="diabatic")
    H = orep.diabatic_h(qmin, qmax, n, wl.NAI_REDUCED_MASS, W, 2)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [5.2], [4.0], [0.35]))
    st = qglib.State(m, precision=qglib.QG_C64_MIXED if prec else qglib.QG_C128)
    st.set(psi0)
    dt = 2.0 if method == 4 else 1.0 * FS
    nsteps = 100 if method == 4 else 2
    st.propagate(method, order, scheme, dt, nsteps, qglib.default_solver_opts(tol=1e-14, solver=solver))
    ora = oprop.DenseStepper(H)
    want = ora.sod(psi0, dt, nsteps)[0] if method == 4 else ora.propagate(psi0, dt, nsteps, method, order, scheme)
    assert rel_l2(st.get(), want) < 1e-11


def test_diabatic_three_states_and_h_psi(qglib, cuda):
    qmin, qmax, n = -6.0, 6.0, 256
    q, dq = ogrid.points(qmin, qmax, n)
    W, dW = _three_state(q)
    g = qglib.Grid([n], [qmin], [qmax])
    m = qglib.Model(g, 3, [50.0], W=W, representation="diabatic")
    H = orep.diabatic_h(qmin, qmax, n, 50.0, W, 3)
    rng = np.random.default_rng(2)
    psi = (rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))) * np.exp(-q ** 2 / 4)
    st = qglib.State(m)
    st.set(psi)
    assert rel_l2(st.apply_h(), (H @ psi.reshape(-1)).reshape(3, n)) < 1e-12
    st.propagate(1, 4, 1, 3.0, 3, qglib.default_solver_opts(tol=1e-14))
    assert rel_l2(st.get(), oprop.DenseStepper(H).propagate(psi, 3.0, 3, 1, 4, 1)) < 1e-11


def test_diabatic_full_size_implicit_equation(qglib, cuda):
    # the NaI-like diabatic model on the paper's grid, one midpoint step at
    # dt = 10.25 a.u.: chi = (psi0 + psi1)/2 solves (1 + i tau H) chi = psi0
    n = 2048
    q, dq = ogrid.points(wl.NAI_QMIN, wl.NAI_QMAX, n)
    W, dW = wl.nai_like_diabatic(q)
    g = qglib.Grid([n], [wl.NAI_QMIN], [wl.NAI_QMAX])
    m = qglib.Model(g, 2, [wl.NAI_REDUCED_MASS], W=W, representation="diabatic")
    H = orep.diabatic_h(wl.NAI_QMIN, wl.NAI_QMAX, n, wl.NAI_REDUCED_MASS, W, 2)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [wl.NAI_Q0], [2.0], [wl.NAI_SIGMA0]))
    st = qglib.State(m)
    st.set(psi0)
    dt = 10500.0 / 1024
    st.propagate(1, 2, 1, dt, 1, qglib.default_solver_opts(tol=1e-15, max_iters=600, solver=1))
    chi = 0.5 * (psi0 + st.get())
    r = chi + 0.5j * dt * (H @ chi.reshape(-1)).reshape(chi.shape) - psi0
    assert np.linalg.norm(r) / np.linalg.norm(psi0) < 1e-13


@pytest.mark.parametrize("S", [2, 3])
def test_representation_change_vs_oracle(qglib, cuda, S):
    qmin, qmax, n = -6.0, 6.0, 512
    q, dq = ogrid.points(qmin, qmax, n)
    W, dW = _two_state(q) if S == 2 else _three_state(q)
    g = qglib.Grid([n], [qmin], [qmax])
    m = qglib.Model(g, S, [100.0], W=W, dW=dW)
    O = orep.rotation(W, S, dW)
    rng = np.random.default_rng(7)
    psi_d = rng.standard_normal((S, n)) + 1j * rng.standard_normal((S, n))
    a = m.to_adiabatic(psi_d)
    np.testing.assert_allclose(a, orep.to_adiabatic(O, psi_d), atol=1e-13)
    np.testing.assert_allclose(m.to_diabatic(a), psi_d, atol=1e-13)
    # device buffers, in place
    t = cuda.tensor(psi_d, device="cuda")
    m.to_adiabatic(t)
    np.testing.assert_allclose(m.to_adiabatic(t).cpu().numpy(), orep.to_adiabatic(O, psi_d), atol=1e-13)


def test_cross_representation_populations_on_the_gpu(qglib, cuda):
    # the same packet propagated in the diabatic and in the adiabatic model
    # (both on the GPU): populations agree to the grid's accuracy (Sec. III)
    qmin, qmax, n, mass = -9.0, 9.0, 512, 400.0
    q, dq = ogrid.points(qmin, qmax, n)
    W, dW = _two_state(q)
    g = qglib.Grid([n], [qmin], [qmax])
    md = qglib.Model(g, 2, [mass], W=W, representation="diabatic")
    ma = qglib.Model(g, 2, [mass], W=W, dW=dW)
    psi_d = oinit.state_on_surface(2, 0, oinit.gaussian([q], [1.5], [0.0], [0.35]))
    sd, sa = qglib.State(md), qglib.State(ma)
    sd.set(psi_d)
    sa.set(ma.to_adiabatic(psi_d))
    opts = qglib.default_solver_opts(tol=1e-14)
    for st in (sd, sa):
        st.propagate(1, 8, 1, 20.0, 20, opts)
    Pa = sa.population()
    Pd = np.sum(np.abs(ma.to_adiabatic(sd.get())) ** 2, axis=1) * dq
    assert min(Pa) > 1e-3
    np.testing.assert_allclose(Pa, Pd, atol=1e-9)


def test_interpolation_vs_oracle(qglib, cuda):
    qmin_s, qmax_s, ns = 3.8, 47.0, 1024
    qmin_d, qmax_d, nd = 3.8 - 2.0, 47.0 + 5.0, 2048
    gs = qglib.Grid([ns], [qmin_s], [qmax_s])
    gd = qglib.Grid([nd], [qmin_d], [qmax_d])
    V = np.zeros((2, ns))
    F = np.zeros((1, 1, ns))
    ms = qglib.Model(gs, 2, [1.0], V=V, F=F)
    md = qglib.Model(gd, 2, [1.0], V=np.zeros((2, nd)), F=np.zeros((1, 1, nd)))
    q, dq = ogrid.points(qmin_s, qmax_s, ns)
    rng = np.random.default_rng(9)
    psi = np.stack([oinit.gaussian([q], [12.0], [3.0], [0.6]), 0.3 * oinit.gaussian([q], [20.0], [-1.0], [1.0])])
    psi = psi + 1e-3 * (rng.standard_normal((2, ns)) + 1j * rng.standard_normal((2, ns)))
    a, b = qglib.State(ms), qglib.State(md)
    a.set(psi)
    b.interpolate_from(a)
    qd, _ = ogrid.points(qmin_d, qmax_d, nd)
    want = orep.trig_interpolate(psi, qmin_s, qmax_s, qd)
    assert rel_l2(b.get(), want) < 1e-11
    # a smooth packet interpolated to a finer grid of the same interval and
    # back to the original points is unchanged
    gf = qglib.Grid([4 * ns], [qmin_s], [qmax_s])
    fine = qglib.State(qglib.Model(gf, 2, [1.0], V=np.zeros((2, 4 * ns)), F=np.zeros((1, 1, 4 * ns))))
    fine.interpolate_from(a)
    back = qglib.State(ms)
    back.interpolate_from(fine)
    assert rel_l2(back.get(), psi) < 1e-12
