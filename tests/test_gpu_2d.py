"""Two-dimensional grids (one instance over the whole GPU, cooperative
launch): H psi, fields and composed steps against the dense oracle on small
grids; at 256 x 256 the complex64-inner / FP64-refined form against the FP64
path, with conservation."""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import FS, rel_l2
from oracle import fields as ofields, grid as ogrid, hamiltonian as oham, initial as oinit, propagate as oprop

pytestmark = pytest.mark.gpu


def _grid_pts(qmin, qmax, ns):
    return [ogrid.points(qmin[d], qmax[d], ns[d])[0] for d in range(2)]


@pytest.mark.parametrize("ns,S", [((16, 16), 2), ((8, 32), 3), ((32, 8), 2)])
def test_hpsi_2d_random_fields_vs_dense_oracle(qglib, cuda, ns, S):
    qmin, qmax, mass = [-3.0, -2.0], [3.0, 2.5], [7.0, 11.0]
    V, F = wl.random_adiabatic_fields(S, 2, ns, seed=40 + S)
    psi = wl.random_psi(S, ns, seed=41 + S)
    g = qglib.Grid(list(ns), qmin, qmax)
    m = qglib.Model(g, S, mass, V=V, F=F)
    st = qglib.State(m)
    st.set(psi)
    got = st.apply_h()
    H = oham.dense_h(qmin, qmax, list(ns), mass, V, F)
    assert rel_l2(got, oham.apply_h(H, psi)) < 1e-12


def _model2d(qg, ns, p=None):
    p = p or wl.MODEL2D_PARAMS
    q1, q2 = _grid_pts(p["qmin"], p["qmax"], ns)
    W, dW = wl.model2d_diabatic(q1, q2, p)
    g = qg.Grid(list(ns), list(p["qmin"]), list(p["qmax"]))
    m = qg.Model(g, 2, list(p["mass"]), W=W, dW=dW)
    return g, m, W, dW, (q1, q2)


def test_fields_2d_vs_oracle(qglib, cuda):
    g, m, W, dW, _ = _model2d(qglib, (64, 32))
    Vg, Fg = m.fields()
    V, F = ofields.two_state(W, dW)
    assert np.abs(Vg - V).max() < 1e-14 * np.abs(V).max() + 1e-17
    assert np.abs(Fg - F).max() < 1e-12 * np.abs(F).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_steps_2d_vs_oracle(qglib, cuda, precision):
    # a smaller, softer copy of the 2-D model on a 16 x 16 grid
    p = dict(wl.MODEL2D_PARAMS, qmin=(-3.0, -2.5), qmax=(3.0, 2.5), mass=(400.0, 400.0))
    ns = (16, 16)
    g, m, W, dW, (q1, q2) = _model2d(qglib, ns, p)
    V, F = ofields.two_state(W, dW)
    H = oham.dense_h(list(p["qmin"]), list(p["qmax"]), list(ns), list(p["mass"]), V, F)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q1, q2], [0.6, 0.1], [1.0, -0.5], [0.5, 0.45]))
    st = qglib.State(m, precision=precision)
    st.set_gaussian(1, [0.6, 0.1], [1.0, -0.5], [0.5, 0.45])
    assert rel_l2(st.get(), psi0) < 1e-13
    dt = 10.0
    s = st.propagate(qglib.QG_MIDPOINT, 6, qglib.QG_SUZUKI, dt, 3, qglib.default_solver_opts(tol=1e-14))
    want = oprop.DenseStepper(H).propagate(psi0, dt, 3, oprop.MIDPOINT, 6, 1)
    err = rel_l2(st.get(), want)
    print("2-D 16x16 Suzuki-6 precision %d: rel L2 vs oracle %.2e (fp64 H psi %d, c64 H psi %d)" %
          (precision, err, s["n_hpsi"], s["n_hpsi32"]))
    assert err < 1e-11
    dv = np.prod([(p["qmax"][d] - p["qmin"][d]) / ns[d] for d in range(2)])
    assert abs(st.norm() - 1.0) < 1e-12
    e_want = (np.vdot(want.reshape(-1), H @ want.reshape(-1)) * dv).real
    assert abs(st.energy() - e_want) < 1e-12 * max(1.0, abs(e_want))


def test_full_size_2d_mixed_vs_fp64(qglib, cuda):
    ns = (256, 256)
    g, m, W, dW, _ = _model2d(qglib, ns)
    q0, p0, s0 = wl.model2d_initial()
    a = qglib.State(m)
    b = qglib.State(m, precision=qglib.QG_C64_MIXED)
    for s in (a, b):
        s.set_gaussian(1, q0, p0, s0)
    e0 = a.energy()
    opts = qglib.default_solver_opts(tol=1e-13)
    sa = a.propagate(qglib.QG_MIDPOINT, 6, qglib.QG_SUZUKI, 0.1 * FS, 3, opts)
    sb = b.propagate(qglib.QG_MIDPOINT, 6, qglib.QG_SUZUKI, 0.1 * FS, 3, opts)
    err = rel_l2(b.get(), a.get())
    print("2-D 256x256 Suzuki-6: mixed vs FP64 rel L2 %.2e; fp64 H psi %d vs %d (+%d c64)" %
          (err, sa["n_hpsi"], sb["n_hpsi"], sb["n_hpsi32"]))
    assert err < 1e-11
    assert abs(a.norm() - 1.0) < 1e-12 and abs(b.norm() - 1.0) < 1e-12
    assert abs(a.energy() - e0) < 1e-12 and abs(b.energy() - e0) < 1e-12
    # plane waves are eigenvectors of the kinetic operator: H e^{ik.q} = k^2/2m e^{ik.q}
    g2 = qglib.Grid(list(ns), [0.0, 0.0], [6.0, 5.0])
    m2 = qglib.Model(g2, 2, [3.0, 5.0], V=np.zeros((2,) + ns), F=np.zeros((2, 1) + ns))
    st = qglib.State(m2)
    q1, q2 = _grid_pts([0.0, 0.0], [6.0, 5.0], ns)
    k1 = ogrid.wavenumbers(0.0, 6.0, ns[0])[7]
    k2 = ogrid.wavenumbers(0.0, 5.0, ns[1])[-3]
    pw = np.exp(1j * (k1 * q1[:, None] + k2 * q2[None, :]))
    st.set(np.stack([pw, 0 * pw]))
    got = st.apply_h()
    want = (k1 ** 2 / 6.0 + k2 ** 2 / 10.0) * pw
    assert np.abs(got[0] - want).max() < 1e-11 * np.abs(want).max()


def test_full_size_2d_hpsi_and_implicit_equation_vs_matrix_free_oracle(qglib, cuda):
    # 256 x 256: H psi element by element against the oracle's 2-D
    # matrix-free H, and one midpoint step of each precision form through its
    # implicit equation (1 + i tau H) chi = psi0, chi = (psi0 + psi1)/2
    ns = (256, 256)
    p = wl.MODEL2D_PARAMS
    g, m, W, dW, (q1, q2) = _model2d(qglib, ns)
    V, F = ofields.two_state(W, dW)
    q0, p0, s0 = wl.model2d_initial()
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q1, q2], q0, [2.0, -1.0], s0))
    h = lambda x: oham.apply_h_matrix_free_2d(list(p["qmin"]), list(p["qmax"]), ns, list(p["mass"]), V, F, x)
    st = qglib.State(m)
    st.set(psi0)
    assert rel_l2(st.apply_h(), h(psi0)) < 1e-12
    dt = 0.5 * FS
    for prec in (qglib.QG_C128, qglib.QG_C64_MIXED):
        s = qglib.State(m, precision=prec)
        s.set(psi0)
        s.propagate(qglib.QG_MIDPOINT, 2, qglib.QG_SUZUKI, dt, 1, qglib.default_solver_opts(tol=1e-14))
        chi = 0.5 * (psi0 + s.get())
        r = chi + 0.5j * dt * h(chi) - psi0
        assert np.linalg.norm(r) / np.linalg.norm(psi0) < 1e-12
