"""Pins of the oracle's dense adiabatic Hamiltonian, Eq. (adiab_mol_ham)."""
import numpy as np
import pytest

import workloads as wl
from oracle import fields, grid, hamiltonian as ham


def test_hermitian_for_random_fields():
    V, F = wl.random_adiabatic_fields(3, 1, (16,), seed=3)
    H = ham.dense_h([0.0], [5.0], [16], [7.0], V, F)
    assert np.abs(H - H.conj().T).max() < 1e-12 * np.abs(H).max()


def test_free_particle_spectrum_is_k2_over_2m():
    n, m = 32, 3.0
    k = grid.wavenumbers(-4.0, 4.0, n)
    H = ham.dense_h([-4.0], [4.0], [n], [m], np.zeros((2, n)), np.zeros((1, 1, n)))
    want = np.sort(np.concatenate([k ** 2 / (2 * m)] * 2))
    np.testing.assert_allclose(np.linalg.eigvalsh(H), want, rtol=0, atol=1e-11 * want.max())


def test_constant_coupling_spectrum_closed_form():
    # F = [[0, c], [-c, 0]] constant: -i hbar F = hbar c sigma_y commutes with p,
    # so A = p +- hbar c on the two eigen-channels and H = (hbar k +- hbar c)^2/2m + v0.
    n, m, c, v0 = 32, 2.5, 0.7, -0.3
    k = grid.wavenumbers(-4.0, 4.0, n)
    V = np.full((2, n), v0)
    F = np.full((1, 1, n), c)
    H = ham.dense_h([-4.0], [4.0], [n], [m], V, F)
    want = np.sort(np.concatenate([(k + c) ** 2 / (2 * m) + v0, (k - c) ** 2 / (2 * m) + v0]))
    np.testing.assert_allclose(np.linalg.eigvalsh(H), want, rtol=0, atol=1e-11)


def _harmonic_two_state(q):
    # two displaced harmonic diabats with a smooth positive coupling (bound spectrum)
    kf, a, d0 = 0.05, 0.6, 0.01
    c, w, c0 = 0.004, 1.0, 0.0015
    w11 = 0.5 * kf * (q - a) ** 2
    w22 = 0.5 * kf * (q + a) ** 2 + d0
    w12 = c * np.exp(-q ** 2 / (2 * w * w)) + c0
    d11 = kf * (q - a)
    d22 = kf * (q + a)
    d12 = -q / (w * w) * c * np.exp(-q ** 2 / (2 * w * w))
    return np.stack([w11, w12, w22]), np.stack([d11, d12, d22])[None]


def test_adiabatic_hamiltonian_has_the_diabatic_spectrum():
    # Sec. II E: the adiabatic H is the diabatic H = p^2/2m + W(q) transformed by
    # O(q); on a converged grid both give the same bound-state energies.  This
    # pins V, the coupling F (and its sign convention), the cross terms and the
    # F^2 term together.
    qmin, qmax, n, m = -9.0, 9.0, 384, 400.0
    q, dq = grid.points(qmin, qmax, n)
    W, dW = _harmonic_two_state(q)
    V, F = fields.two_state(W, dW)
    Ha = ham.dense_h([qmin], [qmax], [n], [m], V, F)
    D = grid.derivative_matrix(qmin, qmax, n)
    T = -(D @ D) / (2 * m)
    Hd = np.kron(np.eye(2), T).astype(complex)
    Hd[:n, :n] += np.diag(W[0])
    Hd[n:, n:] += np.diag(W[2])
    Hd[:n, n:] += np.diag(W[1])
    Hd[n:, :n] += np.diag(W[1])
    ea = np.linalg.eigvalsh(Ha)[:16]
    ed = np.linalg.eigvalsh(Hd)[:16]
    np.testing.assert_allclose(ea, ed, rtol=0, atol=1e-10)
    # a plausible mistake -- dropping the F^2 (diagonal correction) term -- is visible
    Hbad = Ha.copy()
    f2 = F[0, 0] ** 2 / (2 * m)
    Hbad -= np.diag(np.concatenate([f2, f2]))
    assert np.abs(np.linalg.eigvalsh(Hbad)[:16] - ed).max() > 1e-7


def test_matrix_free_action_equals_dense_matrix():
    n = 64
    V, F = wl.random_adiabatic_fields(3, 1, (n,), seed=11)
    psi = wl.random_psi(3, (n,), seed=12)
    H = ham.dense_h([1.0], [9.0], [n], [5.0], V, F)
    a = ham.apply_h(H, psi)
    b = ham.apply_h_matrix_free(1.0, 9.0, n, 5.0, V, F, psi)
    assert np.linalg.norm(a - b) < 1e-12 * np.linalg.norm(a)


def test_two_dimensional_adiabatic_hamiltonian_has_the_diabatic_spectrum():
    # D = 2 (Eq. adiab_mol_ham with a 2-vector of couplings): the adiabatic H
    # built from the two-state fields has the spectrum of p.m^-1.p/2 + W(q)
    p = dict(wl.MODEL2D_PARAMS, qmin=(-3.5, -3.0), qmax=(3.5, 3.0), mass=(400.0, 400.0), c=0.01)
    ns = (32, 32)
    q1 = grid.points(p["qmin"][0], p["qmax"][0], ns[0])[0]
    q2 = grid.points(p["qmin"][1], p["qmax"][1], ns[1])[0]
    W, dW = wl.model2d_diabatic(q1, q2, p)
    V, F = fields.two_state(W, dW)
    Ha = ham.dense_h(list(p["qmin"]), list(p["qmax"]), list(ns), list(p["mass"]), V, F)
    N = ns[0] * ns[1]
    T = np.zeros((N, N), dtype=complex)
    for d in range(2):
        Dd = grid.derivative_along(d, list(p["qmin"]), list(p["qmax"]), list(ns))
        T += -(Dd @ Dd) / (2 * p["mass"][d])
    Hd = np.kron(np.eye(2), T)
    Hd[:N, :N] += np.diag(W[0].reshape(-1))
    Hd[N:, N:] += np.diag(W[2].reshape(-1))
    Hd[:N, N:] += np.diag(W[1].reshape(-1))
    Hd[N:, :N] += np.diag(W[1].reshape(-1))
    np.testing.assert_allclose(np.linalg.eigvalsh(Ha)[:10], np.linalg.eigvalsh(Hd)[:10], rtol=0, atol=5e-8)


@pytest.mark.parametrize("ns,S", [((8, 8), 2), ((12, 16), 3)])
def test_matrix_free_2d_equals_dense(ns, S):
    # the 2-D matrix-free H psi is the dense H of Eq. (adiab_mol_ham) applied
    import workloads as wl
    qmin, qmax, mass = [-3.0, -2.0], [3.0, 2.5], [7.0, 11.0]
    V, F = wl.random_adiabatic_fields(S, 2, ns, seed=60 + S)
    psi = wl.random_psi(S, ns, seed=61 + S)
    H = ham.dense_h(qmin, qmax, list(ns), mass, V, F)
    want = ham.apply_h(H, psi)
    got = ham.apply_h_matrix_free_2d(qmin, qmax, ns, mass, V, F, psi)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-13
