"""Zero initial guess for the implicit solves (QG_GUESS_ZERO) against the
dense oracle and against the explicit-Euler start of Sec. II B: same result
to the solver tolerance, H psi accounting, 2-D and adjoint forms."""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import FS, nai_library_model, nai_oracle_fields, rel_l2
from oracle import grid as ogrid, hamiltonian as oham, initial as oinit, propagate as oprop

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method,order,scheme,precision,solver",
                         [(0, 2, 0, 0, 0), (1, 4, 1, 0, 1), (0, 6, 0, 0, 1), (1, 8, 1, 0, 0), (1, 6, 1, 1, 1),
                          (0, 4, 0, 1, 0)])
def test_zero_guess_vs_oracle(qglib, cuda, method, order, scheme, precision, solver):
    qmin, qmax, n = 3.8, 12.0, 128
    grid, model = nai_library_model(qglib, n, qmin, qmax)
    V, F = nai_oracle_fields(n, qmin, qmax)
    H = oham.dense_h([qmin], [qmax], [n], [wl.NAI_REDUCED_MASS], V, F)
    q, dq = ogrid.points(qmin, qmax, n)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [5.2], [4.0], [0.35]))
    st = qglib.State(model, precision=precision)
    st.set(psi0)
    opts = qglib.default_solver_opts(tol=1e-14, solver=solver, guess=qglib.QG_GUESS_ZERO, true_residual=1)
    s = st.propagate(method, order, scheme, 1.0 * FS, 2, opts)
    want = oprop.DenseStepper(H).propagate(psi0, 1.0 * FS, 2, method, order, scheme)
    err = rel_l2(st.get(), want)
    print("zero guess vs oracle (method %d order %d scheme %d precision %d solver %d): %.2e" %
          (method, order, scheme, precision, solver, err))
    assert err < 1e-11


@pytest.mark.parametrize("solver", [0, 1])
def test_zero_guess_equals_euler_guess_full_size(qglib, cuda, solver):
    # the bench operating point: N = 2048, midpoint, Suzuki 8, dt = 10.25 a.u., tol 1e-15
    n = 2048
    grid, model = nai_library_model(qglib, n)
    a, b = qglib.State(model), qglib.State(model)
    for s in (a, b):
        s.set_gaussian(1, [wl.NAI_Q0], [wl.NAI_P0], [wl.NAI_SIGMA0])
    dt = 10500.0 / 1024
    sa = a.propagate(1, 8, 1, dt, 2, qglib.default_solver_opts(tol=1e-15, solver=solver))
    sb = b.propagate(1, 8, 1, dt, 2, qglib.default_solver_opts(tol=1e-15, solver=solver, guess=qglib.QG_GUESS_ZERO))
    err = rel_l2(b.get(), a.get())
    print("solver %d: zero vs Euler guess %.2e; H psi per sub-step %.3f (zero) vs %.3f (Euler)" %
          (solver, err, sb["n_hpsi"] / sb["n_substeps"], sa["n_hpsi"] / sa["n_substeps"]))
    assert err < 1e-12
    # midpoint with the 2 chi - psi epilogue: one H psi per Krylov iteration
    # and per restart, none for the guess or the first residual
    assert sb["n_hpsi"] == sb["n_krylov"] + sb["n_restart"]
    # Euler start: H psi carried between sub-steps, one exact H psi per
    # composed step (2 here), then the residual of the start
    assert sa["n_hpsi"] == 2 + sa["n_substeps"] + sa["n_krylov"] + sa["n_restart"]
    assert abs(b.norm() - 1.0) < 1e-12


def test_zero_guess_trapezoidal_counts(qglib, cuda):
    # trapezoidal rule: b = (1 - i tau H) psi costs one H psi per sub-step
    grid, model = nai_library_model(qglib, 1024)
    st = qglib.State(model)
    st.set_gaussian(1, [wl.NAI_Q0], [wl.NAI_P0], [wl.NAI_SIGMA0])
    s = st.propagate(0, 4, 1, 0.5 * FS, 3,
                     qglib.default_solver_opts(tol=1e-13, solver=1, guess=qglib.QG_GUESS_ZERO))
    assert s["n_hpsi"] == s["n_substeps"] + s["n_krylov"] + s["n_restart"]


def test_zero_guess_2d(qglib, cuda):
    p = wl.MODEL2D_PARAMS
    ns = (128, 64)
    q1 = ogrid.points(p["qmin"][0], p["qmax"][0], ns[0])[0]
    q2 = ogrid.points(p["qmin"][1], p["qmax"][1], ns[1])[0]
    W, dW = wl.model2d_diabatic(q1, q2, p)
    g = qglib.Grid(list(ns), list(p["qmin"]), list(p["qmax"]))
    m = qglib.Model(g, 2, list(p["mass"]), W=W, dW=dW)
    q0, p0, s0 = wl.model2d_initial()
    out = {}
    for prec in (0, 1):
        for guess in (0, 1):
            st = qglib.State(m, precision=prec)
            st.set_gaussian(1, q0, p0, s0)
            st.propagate(1, 6, 1, 0.1 * FS, 2, qglib.default_solver_opts(tol=1e-13, solver=1, guess=guess))
            out[prec, guess] = st.get()
    ref = out[0, 0]
    for k, v in out.items():
        err = rel_l2(v, ref)
        print("2-D 128x64 precision %d guess %d vs FP64 Euler start: %.2e" % (k[0], k[1], err))
        assert err < 1e-11


def test_zero_guess_adjoint_identity(qglib, cuda):
    torch = cuda
    from paper_1902_04661_gb300 import autograd as qad
    n = 256
    qmin, qmax = 3.8, 14.0
    grid, model = nai_library_model(qglib, n, qmin, qmax)
    V, F = nai_oracle_fields(n, qmin, qmax)
    q, dq = ogrid.points(qmin, qmax, n)
    psi0 = oinit.state_on_surface(2, 1, oinit.gaussian([q], [5.0], [2.0], [0.3]))
    rng = np.random.default_rng(11)
    lam = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    grads = {}
    for guess in (0, 1):
        opts = qglib.default_solver_opts(tol=1e-15, solver=1, guess=guess)
        Vt = torch.tensor(V, device="cuda", requires_grad=True)
        Ft = torch.tensor(F[0], device="cuda", requires_grad=True)
        p0 = torch.tensor(psi0, device="cuda", requires_grad=True)
        out = qad.propagate(Vt, Ft, p0, grid, wl.NAI_REDUCED_MASS, 1, 4, 1, 1.0 * FS, 6, 2, opts)
        L = (torch.tensor(lam, device="cuda").conj() * out).sum().real
        L.backward()
        grads[guess] = (Vt.grad.cpu().numpy(), Ft.grad.cpu().numpy(), p0.grad.cpu().numpy())
    for a, b in zip(grads[0], grads[1]):
        assert np.abs(a - b).max() < 1e-9 * max(1.0, np.abs(a).max())
