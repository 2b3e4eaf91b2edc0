"""Pins of the oracle's integrators (Secs. II A-C, Theorem, Appendix A)."""
import numpy as np
import pytest

import workloads as wl
from oracle import composition as comp, grid, hamiltonian as ham, initial, observables as obs, propagate as prop


@pytest.fixture(scope="module")
def small():
    qmin, qmax, n = 3.8, 12.0, 48
    q, dq = grid.points(qmin, qmax, n)
    W, dW = wl.nai_like_diabatic(q)
    from oracle import fields
    V, F = fields.two_state(W, dW)
    H = ham.dense_h([qmin], [qmax], [n], [wl.NAI_REDUCED_MASS], V, F)
    psi = initial.state_on_surface(2, 1, initial.gaussian([q], [5.5], [3.0], [0.45]))
    phi = initial.state_on_surface(2, 1, initial.gaussian([q], [6.0], [-2.5], [0.45]))
    return dict(H=H, psi=psi, phi=phi, dq=dq)


@pytest.mark.parametrize("order,scheme", [(2, 0), (4, 0), (4, 1), (6, 1), (8, 0)])
def test_trapezoidal_equals_midpoint(small, order, scheme):
    # Proposition 2 / Appendix A: the Cayley factors commute for a
    # time-independent H, so both rules give the same map
    st = prop.DenseStepper(small["H"])
    a = st.propagate(small["psi"], 30.0, 3, prop.TRAPEZOIDAL, order, scheme)
    b = st.propagate(small["psi"], 30.0, 3, prop.MIDPOINT, order, scheme)
    assert np.linalg.norm(a - b) < 1e-12


@pytest.mark.parametrize("order,scheme", [(2, 1), (4, 0), (6, 0), (8, 1)])
def test_lu_route_equals_eigen_route(small, order, scheme):
    st = prop.DenseStepper(small["H"])
    a = st.propagate(small["psi"], 25.0, 2, prop.MIDPOINT, order, scheme)
    b = prop.cayley_by_eigen(small["H"], small["psi"], 25.0, comp.schedule(order, scheme), 2)
    assert np.linalg.norm(a - b) < 1e-12


def test_invariants_conserved(small):
    # Theorem (Sec. II C): norm, inner product, symplectic form and energy
    H, dq = small["H"], small["dq"]
    st = prop.DenseStepper(H)
    psi, phi = small["psi"], small["phi"]
    n0, e0, w0, s0 = obs.norm(psi, dq), obs.energy(H, psi, dq), obs.omega(psi, phi, dq), obs.inner(psi, phi, dq)
    a, b = psi, phi
    for _ in range(20):
        a = st.composed(a, 50.0, prop.TRAPEZOIDAL, 4, comp.SUZUKI)
        b = st.composed(b, 50.0, prop.TRAPEZOIDAL, 4, comp.SUZUKI)
    assert abs(obs.norm(a, dq) - n0) < 1e-13
    assert abs(obs.energy(H, a, dq) - e0) < 1e-13 * max(1.0, np.abs(H).max())
    assert abs(obs.omega(a, b, dq) - w0) < 1e-13
    assert abs(obs.inner(a, b, dq) - s0) < 1e-13


def test_time_reversibility(small):
    # U(-t) U(t) psi = psi for the symmetric compositions
    st = prop.DenseStepper(small["H"])
    a = st.propagate(small["psi"], 40.0, 10, prop.MIDPOINT, 6, comp.SUZUKI)
    b = st.propagate(a, -40.0, 10, prop.MIDPOINT, 6, comp.SUZUKI)
    assert np.linalg.norm(b - small["psi"]) * np.sqrt(small["dq"]) < 1e-12


def test_euler_methods_are_not_unitary(small):
    # Sec. II B: explicit Euler grows the norm, implicit Euler shrinks it
    st = prop.DenseStepper(small["H"])
    dq = small["dq"]
    assert obs.norm(st.expl(small["psi"], 5.0), dq) > 1.0 + 1e-6
    assert obs.norm(st.impl(small["psi"], 5.0), dq) < 1.0 - 1e-6


@pytest.mark.parametrize("order,scheme,ns", [(2, 0, (16, 32)), (4, 0, (16, 32)), (4, 1, (8, 16)),
                                             (6, 0, (16, 32)), (6, 1, (4, 8)), (8, 0, (16, 32)), (8, 1, (3, 6))])
def test_global_error_order_against_exact_evolution(order, scheme, ns):
    # Table I / Fig. 3: global error O(dt^order) against e^{-iHt}
    rng = np.random.default_rng(5)
    A = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    H = (A + A.conj().T) / 8.0
    psi = rng.standard_normal(12) + 0j
    psi /= np.linalg.norm(psi)
    t = 6.0 if (order, scheme) == (8, 1) else 2.0
    ex = prop.exact(H, psi, t)
    st = prop.DenseStepper(H)
    err = []
    for n in ns:
        err.append(np.linalg.norm(st.propagate(psi, t / n, n, prop.MIDPOINT, order, scheme) - ex))
    slope = np.log(err[0] / err[1]) / np.log(2.0)
    assert abs(slope - order) < 0.35, (err, slope)


@pytest.mark.parametrize("method", [prop.TRAPEZOIDAL, prop.MIDPOINT])
def test_columns_route_equals_one_state_route(small, method):
    # several states through one LU solve with many right-hand sides give
    # the states propagated one by one
    st = prop.DenseStepper(small["H"])
    many = st.propagate_columns([small["psi"], small["phi"]], 30.0, 2, method, 6, comp.SUZUKI)
    for got, psi in zip(many, (small["psi"], small["phi"])):
        want = st.propagate(psi, 30.0, 2, method, 6, comp.SUZUKI)
        assert np.linalg.norm(got - want) < 1e-12


def test_cached_exact_evolution_equals_exact(small):
    ev = prop.ExactEvolution(small["H"])
    for t in (0.0, 37.5, -120.0):
        assert np.linalg.norm(ev(small["psi"], t) - prop.exact(small["H"], small["psi"], t)) < 1e-12
