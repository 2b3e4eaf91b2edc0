"""Adjoint form: reverse-mode gradients through the composed implicit
propagation by time-reversed re-propagation (torch.autograd.Function over the
library's adjoint kernel), checked against central finite differences of the
dense oracle, the adjoint identity, and finite differences at full size."""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import FS, rel_l2
from oracle import fields as ofields, grid as ogrid, hamiltonian as oham, initial as oinit, propagate as oprop

pytestmark = pytest.mark.gpu

SMALL = (3.8, 12.0, 64)


def _setup_small(torch, qg):
    qmin, qmax, n = SMALL
    q, dq = ogrid.points(qmin, qmax, n)
    W, dW = wl.nai_like_diabatic(q)
    V, F = ofields.two_state(W, dW)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [5.6], [3.0], [0.45]))
    grid = qg.Grid([n], [qmin], [qmax])
    return grid, V, F, psi0, dq


def _oracle_loss(V, F, psi0, dq, kind, nsteps, dt):
    qmin, qmax, n = SMALL
    H = oham.dense_h([qmin], [qmax], [n], [wl.NAI_REDUCED_MASS], V, F)
    psi = oprop.DenseStepper(H).propagate(psi0, dt, nsteps, oprop.MIDPOINT, 4, 1)
    if kind == "pop":
        return dq * np.sum(np.abs(psi[1]) ** 2)
    return (dq * np.vdot(psi0, psi)).real


@pytest.mark.parametrize("kind", ["pop", "autocorr"])
def test_adjoint_gradients_vs_oracle_finite_differences(qglib, cuda, kind):
    torch = cuda
    from paper_1902_04661_gb300 import autograd as qad
    grid, V, F, psi0, dq = _setup_small(torch, qglib)
    dt, nsteps = 1.0 * FS, 6
    opts = qglib.default_solver_opts(tol=1e-14)
    Vt = torch.tensor(V, device="cuda", requires_grad=True)
    Ft = torch.tensor(F[0], device="cuda", requires_grad=True)
    p0 = torch.tensor(psi0, device="cuda", requires_grad=True)
    out = qad.propagate(Vt, Ft, p0, grid, wl.NAI_REDUCED_MASS, qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, dt, nsteps,
                        2, opts)
    if kind == "pop":
        L = dq * (out[1].abs() ** 2).sum()
    else:
        L = (dq * (p0.conj() * out).sum()).real
    L.backward()
    gV, gF, g0 = Vt.grad.cpu().numpy(), Ft.grad.cpu().numpy(), p0.grad.cpu().numpy()
    L0 = _oracle_loss(V, F, psi0, dq, kind, nsteps, dt)
    assert abs(L.item() - L0) < 1e-12
    h = 1e-6
    rng = np.random.default_rng(3)
    for _ in range(6):
        s, j = int(rng.integers(0, 2)), int(rng.integers(8, 56))
        Vp, Vm = V.copy(), V.copy()
        Vp[s, j] += h
        Vm[s, j] -= h
        fd = (_oracle_loss(Vp, F, psi0, dq, kind, nsteps, dt) - _oracle_loss(Vm, F, psi0, dq, kind, nsteps, dt)) / (2 * h)
        assert abs(gV[s, j] - fd) < 1e-7 * max(1.0, abs(fd)), (s, j, gV[s, j], fd)
        Fp, Fm = F.copy(), F.copy()
        Fp[0, 0, j] += h
        Fm[0, 0, j] -= h
        fd = (_oracle_loss(V, Fp, psi0, dq, kind, nsteps, dt) - _oracle_loss(V, Fm, psi0, dq, kind, nsteps, dt)) / (2 * h)
        assert abs(gF[0, j] - fd) < 1e-7 * max(1.0, abs(fd)), (j, gF[0, j], fd)
        for comp, unit in ((0, 1.0), (1, 1j)):
            pp, pm = psi0.copy(), psi0.copy()
            pp[1, j] += h * unit
            pm[1, j] -= h * unit
            fd = (_oracle_loss(V, F, pp, dq, kind, nsteps, dt) - _oracle_loss(V, F, pm, dq, kind, nsteps, dt)) / (2 * h)
            got = g0[1, j].real if comp == 0 else g0[1, j].imag
            assert abs(got - fd) < 1e-7 * max(1.0, abs(fd)), (j, comp, got, fd)


def test_adjoint_identity_and_reconstruction(qglib, cuda):
    torch = cuda
    import ctypes
    grid, V, F, psi0, dq = _setup_small(torch, qglib)
    n = SMALL[2]
    model = qglib.Model(grid, 2, [wl.NAI_REDUCED_MASS], V=V, F=F)
    st = qglib.State(model)
    st.set(psi0)
    every, nsteps = 3, 7
    nck = (nsteps - 1) // every + 1
    ck = torch.empty((nck, 2, n), dtype=torch.complex128, device="cuda")
    lam = torch.tensor(wl.random_psi(2, (n,), seed=9, smooth=12), device="cuda")
    g = lam.clone()
    gV = torch.zeros((2, n), dtype=torch.float64, device="cuda")
    gF = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    assert qglib.lib().qg_state_set_adjoint(st.handle, P(ck), nck, every, P(g), P(gV), P(gF)) == 0
    opts = qglib.default_solver_opts(tol=1e-14)
    o = qglib.StepStats()
    assert qglib.lib().qg_propagate_ex(st.handle, 1, 0, 6, 1, 0.7 * FS, nsteps, ctypes.byref(opts), ctypes.byref(o)) == 0
    upsi = st.get()
    assert qglib.lib().qg_propagate_ex(st.handle, 2, 0, 6, 1, 0.7 * FS, nsteps, ctypes.byref(opts), ctypes.byref(o)) == 0
    # <lambda|U psi> = <U^dagger lambda|psi>, up to the solver accuracy: 63
    # forward and 126 backward solves, each exact to its residual
    lhs = np.vdot(lam.cpu().numpy(), upsi)
    rhs = np.vdot(g.cpu().numpy(), psi0)
    assert abs(lhs - rhs) < 2e-10 * abs(lhs)
    # the backward run ends on the checkpoint of step 0, i.e. psi0 itself
    np.testing.assert_array_equal(st.get(), psi0)


def test_batched_adjoint_equals_single(qglib, cuda):
    torch = cuda
    from paper_1902_04661_gb300 import autograd as qad
    grid, V, F, psi0, dq = _setup_small(torch, qglib)
    opts = qglib.default_solver_opts(tol=1e-13)
    Bn = 3
    Vb = torch.tensor(np.stack([V * (1 + 0.01 * b) for b in range(Bn)]), device="cuda", requires_grad=True)
    Fb = torch.tensor(np.stack([F[0] * (1 - 0.02 * b) for b in range(Bn)]), device="cuda", requires_grad=True)
    pb = torch.tensor(np.stack([psi0] * Bn), device="cuda", requires_grad=True)
    out = qad.propagate_batch(Vb, Fb, pb, grid, wl.NAI_REDUCED_MASS, 1, 4, 1, 0.5 * FS, 4, 2, opts)
    (out[:, 1].abs() ** 2).sum().backward()
    for b in range(Bn):
        v = Vb[b].detach().clone().requires_grad_(True)
        f = Fb[b].detach().clone().requires_grad_(True)
        p = pb[b].detach().clone().requires_grad_(True)
        o1 = qad.propagate(v, f, p, grid, wl.NAI_REDUCED_MASS, 1, 4, 1, 0.5 * FS, 4, 2, opts)
        (o1[1].abs() ** 2).sum().backward()
        np.testing.assert_array_equal(o1.detach().cpu().numpy(), out[b].detach().cpu().numpy())
        np.testing.assert_array_equal(v.grad.cpu().numpy(), Vb.grad[b].cpu().numpy())
        np.testing.assert_array_equal(f.grad.cpu().numpy(), Fb.grad[b].cpu().numpy())
        np.testing.assert_array_equal(p.grad.cpu().numpy(), pb.grad[b].cpu().numpy())


THETA = ["E_ion", "A_ion", "rho_ion", "B_cov", "rho_cov", "A_c", "beta_c", "q_c"]


def test_full_size_parameter_gradients_vs_central_differences(qglib, cuda):
    # N = 2048 NaI-like model, order-4 Suzuki midpoint: gradients of the
    # population transferred to the ground state by a packet launched through
    # the avoided crossing, with respect to the 8 diabatic parameters and the
    # Gaussian's q0, p0, against central differences (h = 1e-6, relative to
    # each parameter) of the full GPU propagation
    torch = cuda
    from paper_1902_04661_gb300 import autograd as qad
    n = 2048
    grid = qglib.Grid([n], [wl.NAI_QMIN], [wl.NAI_QMAX])
    q = grid.points()
    dq = grid.dq[0]
    base = wl.nai_like_params()
    q0, p0, s0 = 12.9, 20.0, 0.3
    dt, nsteps = 1.0 * FS, 20
    opts = qglib.default_solver_opts(tol=1e-14)

    def fields(par):
        W, dW = wl.nai_like_diabatic(q, par)
        m = qglib.Model(grid, 2, [wl.NAI_REDUCED_MASS], W=W, dW=dW)
        return m.fields()

    def gauss(qq, pp):
        st = qglib.State(qglib.Model(grid, 2, [1.0], V=np.zeros((2, n)), F=np.zeros((1, 1, n))))
        st.set_gaussian(1, [qq], [pp], [s0])
        return st.get()

    def loss(par, qq, pp):
        V, F = fields(par)
        m = qglib.Model(grid, 2, [wl.NAI_REDUCED_MASS], V=V, F=F)
        st = qglib.State(m)
        st.set(gauss(qq, pp))
        st.propagate(1, 4, 1, dt, nsteps, opts)
        return st.population()[0]

    V, F = fields(base)
    Vt = torch.tensor(V, device="cuda", requires_grad=True)
    Ft = torch.tensor(F[0], device="cuda", requires_grad=True)
    pt = torch.tensor(gauss(q0, p0), device="cuda", requires_grad=True)
    out = qad.propagate(Vt, Ft, pt, grid, wl.NAI_REDUCED_MASS, 1, 4, 1, dt, nsteps, 4, opts)
    L = dq * (out[0].abs() ** 2).sum()
    L.backward()
    assert L.item() > 1e-4          # the packet really crosses
    gV, gF, g0 = Vt.grad.cpu().numpy(), Ft.grad.cpu().numpy(), pt.grad.cpu().numpy()
    hr = 1e-6
    pairs = []
    for name in THETA:
        h = hr * abs(base[name])
        bp, bm = dict(base), dict(base)
        bp[name] += h
        bm[name] -= h
        Vp, Fp = fields(bp)
        Vm, Fm = fields(bm)
        dVdt = (Vp - Vm) / (2 * h)
        dFdt = (Fp[0] - Fm[0]) / (2 * h)
        adj = float(np.sum(gV * dVdt) + np.sum(gF * dFdt))
        fd = (loss(bp, q0, p0) - loss(bm, q0, p0)) / (2 * h)
        # noise floor of the difference quotient: each loss is exact to about
        # the solver tolerance, so fd carries ~ 1e-13 / (2 h)
        pairs.append((name, adj, fd, 1e-13 / (2 * h)))
    for which in ("q0", "p0"):
        h = 1e-6
        a = (q0 + h, p0) if which == "q0" else (q0, p0 + h)
        b = (q0 - h, p0) if which == "q0" else (q0, p0 - h)
        dpsi = (gauss(*a) - gauss(*b)) / (2 * h)
        adj = float(np.sum((np.conj(g0) * dpsi).real))
        fd = (loss(base, *a) - loss(base, *b)) / (2 * h)
        pairs.append((which, adj, fd, 1e-13 / (2 * h)))
    for name, adj, fd, noise in pairs:
        assert abs(adj - fd) < 1e-5 * abs(fd) + noise, (name, adj, fd, noise)
