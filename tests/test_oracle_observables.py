"""Pins of the oracle's observables (Sec. II A) against closed forms.

Each pin uses a grid spacing far from 1, so a dropped volume element fails,
and puts different values on different surfaces, so a swapped surface index
fails:

* populations: a packet loaded on one surface gives (0, 1); an uneven split
  a psi on surface 0, b psi on surface 1 gives (|a|^2, |b|^2);
* energy: a free Gaussian (V = F = 0) has <H> = p0^2/2m + 1/(8 m sigma0^2);
  the ground state of V_s = m w^2 (q - qc)^2 / 2 + v_s has <H> = w/2 + v_s;
* omega = -2 hbar Im<psi|phi> (Eq. def_symplectic_two_form) of two Gaussians
  of equal width:
  <psi_a|psi_b> = exp(-(qa - qb)^2/(8 s^2) - s^2 (pb - pa)^2/2)
                  * exp(i (pa + pb)(qa - qb)/2).
"""
import numpy as np
import pytest

from oracle import grid, hamiltonian as ham, initial, observables as obs


def _gauss_overlap(qa, pa, qb, pb, s):
    mag = np.exp(-(qa - qb) ** 2 / (8.0 * s * s) - s * s * (pb - pa) ** 2 / 2.0)
    return mag * np.exp(1j * (pa + pb) * (qa - qb) / 2.0)


@pytest.fixture(scope="module")
def line():
    qmin, qmax, n = -12.0, 12.0, 128
    q, dq = grid.points(qmin, qmax, n)
    assert abs(dq - 0.1875) < 1e-15
    return qmin, qmax, n, q, dq


def test_populations_single_surface_and_split(line):
    qmin, qmax, n, q, dq = line
    g = initial.gaussian([q], [0.7], [0.4], [1.1])
    psi = initial.state_on_surface(2, 1, g)
    P = obs.populations(psi, dq)
    assert abs(P[0]) < 1e-15 and abs(P[1] - 1.0) < 1e-13
    a, b = np.sqrt(0.3), np.sqrt(0.7) * np.exp(0.4j)
    split = np.stack([a * g, b * g])
    P = obs.populations(split, dq)
    assert abs(P[0] - 0.3) < 1e-13 and abs(P[1] - 0.7) < 1e-13
    assert abs(obs.norm(split, dq) - 1.0) < 1e-13


def test_energy_of_free_gaussian(line):
    qmin, qmax, n, q, dq = line
    m, q0, p0, s0 = 1.7, 0.5, 1.5, 1.0
    V = np.zeros((2, n))
    F = np.zeros((1, 1, n))
    H = ham.dense_h([qmin], [qmax], [n], [m], V, F)
    psi = initial.state_on_surface(2, 1, initial.gaussian([q], [q0], [p0], [s0]))
    E = obs.energy(H, psi, dq)
    assert abs(E - (p0 ** 2 / (2 * m) + 1.0 / (8 * m * s0 ** 2))) < 1e-12


def test_energy_of_harmonic_ground_state_on_one_surface(line):
    qmin, qmax, n, q, dq = line
    m, w, qc = 2.0, 0.5, 0.3
    s0 = np.sqrt(1.0 / (2.0 * m * w))     # std-dev of |psi|^2 in the ground state
    v = (0.25, -0.125)                    # surface offsets: a swapped index fails
    V = np.stack([0.5 * m * w * w * (q - qc) ** 2 + v[0], 0.5 * m * w * w * (q - qc) ** 2 + v[1]])
    F = np.zeros((1, 1, n))
    H = ham.dense_h([qmin], [qmax], [n], [m], V, F)
    for s in (0, 1):
        psi = initial.state_on_surface(2, s, initial.gaussian([q], [qc], [0.0], [s0]))
        assert abs(obs.energy(H, psi, dq) - (w / 2 + v[s])) < 1e-12
        # it is an eigenstate: H psi = E psi on the grid to spectral accuracy
        Hpsi = ham.apply_h(H, psi)
        assert np.linalg.norm(Hpsi - (w / 2 + v[s]) * psi) * np.sqrt(dq) < 1e-10


def test_inner_product_and_omega_of_two_gaussians(line):
    qmin, qmax, n, q, dq = line
    s = 0.9
    qa, pa, qb, pb = -1.0, 0.8, 0.6, -0.5
    ga = initial.gaussian([q], [qa], [pa], [s])
    gb = initial.gaussian([q], [qb], [pb], [s])
    psi = initial.state_on_surface(2, 1, ga)
    phi = initial.state_on_surface(2, 1, gb)
    ref = _gauss_overlap(qa, pa, qb, pb, s)
    assert abs(obs.inner(psi, phi, dq) - ref) < 1e-12
    w = obs.omega(psi, phi, dq)
    assert abs(w - (-2.0 * ref.imag)) < 1e-12
    assert abs(w) > 0.1                        # the pin is not a trivial zero
    # antisymmetry of the two-form (a conjugated wrong argument fails)
    assert abs(obs.omega(phi, psi, dq) + w) < 1e-12
    # components on different surfaces do not overlap
    psi0 = initial.state_on_surface(2, 0, ga)
    assert abs(obs.omega(psi0, phi, dq)) < 1e-15
    # both surfaces loaded: the overlaps add per surface
    two_a = np.stack([ga, 2.0 * ga]) / np.sqrt(5.0)
    two_b = np.stack([gb, -gb]) / np.sqrt(2.0)
    ref2 = (1.0 - 2.0) / np.sqrt(10.0) * ref
    assert abs(obs.inner(two_a, two_b, dq) - ref2) < 1e-12
