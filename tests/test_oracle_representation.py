"""Pins of the oracle's diabatic representation (Sec. II E) and of the
trigonometric interpolation between grids (Appendix B).

* the diabatic H of a constant W has the spectrum k^2/2m + eig(W) (kinetic
  term, W blocks and their placement);
* O^T W O = diag(V ascending) at every point, O orthogonal (pins the
  transform's orientation and the surface order);
* the diabatic and the adiabatic H of one model share their bound spectrum on
  a converged grid, and the same packet evolved exactly in either
  representation gives the same adiabatic populations -- the
  cross-representation check of Sec. III;
* interpolation reproduces trigonometric polynomials exactly, real data
  stays real, a Gaussian converges fast with the density of the source grid.
"""
import numpy as np
import pytest

from oracle import fields, grid, hamiltonian as ham, initial, propagate as prop, representation as rep


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


def test_constant_w_spectrum():
    n, m = 32, 2.0
    k = grid.wavenumbers(-5.0, 5.0, n)
    Wc = np.array([[0.3, 0.1], [0.1, -0.2]])
    W = np.stack([np.full(n, Wc[0, 0]), np.full(n, Wc[0, 1]), np.full(n, Wc[1, 1])])
    H = rep.diabatic_h(-5.0, 5.0, n, m, W, 2)
    want = np.sort(np.concatenate([k ** 2 / (2 * m) + e for e in np.linalg.eigvalsh(Wc)]))
    np.testing.assert_allclose(np.linalg.eigvalsh(H), want, rtol=0, atol=1e-12)
    assert np.abs(H - H.conj().T).max() < 1e-13


@pytest.mark.parametrize("S", [2, 3])
def test_rotation_diagonalises_w(S):
    q, dq = grid.points(-6.0, 6.0, 64)
    if S == 2:
        W, dW = _two_state(q)
        V, F = fields.two_state(W, dW)
    else:
        rng = np.random.default_rng(4)
        A = rng.standard_normal((6, 3))
        W = np.stack([A[t, 0] + A[t, 1] * np.sin(q) + A[t, 2] * q * 0.1 for t in range(6)]) * 0.1
        dW = np.stack([A[t, 1] * np.cos(q) + A[t, 2] * 0.1 for t in range(6)])[None] * 0.1
        V, F, _ = fields.general_adiabatic(W, dW, 3)
    O = rep.rotation(W, S, dW)
    Wm = fields.unpack_symmetric(W, S)
    for j in range(0, 64, 7):
        np.testing.assert_allclose(O[j].T @ O[j], np.eye(S), atol=1e-14)
        np.testing.assert_allclose(O[j].T @ Wm[j] @ O[j], np.diag(V[:, j]), atol=1e-13)
    # the coupling F = O^T O' (Sec. II E) with the library's sign convention:
    # F[0] = <ground | d/dq excited>
    if S == 2:
        h = 1e-5
        dO = (rep.rotation(_two_state(q + h)[0], 2) - rep.rotation(_two_state(q - h)[0], 2)) / (2 * h)
        f = np.einsum("jr,jr->j", O[:, :, 0], dO[:, :, 1])
        np.testing.assert_allclose(f, F[0, 0], atol=1e-7)


def test_transform_round_trip_and_norm():
    q, dq = grid.points(-6.0, 6.0, 64)
    W, dW = _two_state(q)
    O = rep.rotation(W, 2)
    rng = np.random.default_rng(1)
    psi = rng.standard_normal((2, 64)) + 1j * rng.standard_normal((2, 64))
    a = rep.to_adiabatic(O, psi)
    assert abs(np.linalg.norm(a) - np.linalg.norm(psi)) < 1e-12
    np.testing.assert_allclose(rep.to_diabatic(O, a), psi, atol=1e-13)


def _cross(n, t=400.0):
    qmin, qmax, m = -9.0, 9.0, 400.0
    q, dq = grid.points(qmin, qmax, n)
    W, dW = _two_state(q)
    Hd = rep.diabatic_h(qmin, qmax, n, m, W, 2)
    Ha = rep.adiabatic_h_from_diabatic(qmin, qmax, n, m, W, dW)
    O = rep.rotation(W, 2)
    psi_d = initial.state_on_surface(2, 0, initial.gaussian([q], [1.5], [0.0], [0.35]))
    a_from_d = rep.to_adiabatic(O, prop.exact(Hd, psi_d, t))
    a_direct = prop.exact(Ha, rep.to_adiabatic(O, psi_d), t)
    Pa = np.sum(np.abs(a_direct) ** 2, axis=1) * dq
    Pd = np.sum(np.abs(a_from_d) ** 2, axis=1) * dq
    return Hd, Ha, Pa, Pd


def test_cross_representation_spectrum_and_populations():
    # the two representations differ on the grid only by discretisation:
    # bound energies agree and the populations converge exponentially with
    # the grid density (Appendix B)
    Hd, Ha, Pa, Pd = _cross(384)
    np.testing.assert_allclose(np.linalg.eigvalsh(Ha)[:12], np.linalg.eigvalsh(Hd)[:12], rtol=0, atol=1e-9)
    assert min(Pa) > 1e-3                     # population has moved between surfaces
    np.testing.assert_allclose(Pa, Pd, atol=1e-10)
    _, _, Pa2, Pd2 = _cross(256)
    assert np.abs(Pa2 - Pd2).max() > 100 * np.abs(Pa - Pd).max()


def test_trig_interpolation():
    qmin, qmax, n = -3.0, 5.0, 32
    q, dq = grid.points(qmin, qmax, n)
    L = qmax - qmin
    f = lambda x: (np.exp(2j * np.pi * 3 * (x - qmin) / L) + 0.5 * np.cos(2 * np.pi * 7 * (x - qmin) / L)
                   - 0.25j * np.sin(2 * np.pi * 15 * (x - qmin) / L))
    qo = np.linspace(qmin, qmax, 97, endpoint=False) + 0.013
    np.testing.assert_allclose(rep.trig_interpolate(f(q), qmin, qmax, qo), f(qo), atol=1e-13)
    # the Nyquist cosine: a real sample set gives a real interpolant
    g = np.cos(np.pi * (q - qmin) / dq)
    assert np.abs(rep.trig_interpolate(g, qmin, qmax, qo).imag).max() < 1e-13
    # a Gaussian converges quickly with the source density
    gau = lambda x: np.exp(-(x - 1.0) ** 2 / 0.5)
    errs = []
    for ns in (16, 24, 32):
        qs, _ = grid.points(qmin, qmax, ns)
        errs.append(np.abs(rep.trig_interpolate(gau(qs), qmin, qmax, qo) - gau(qo)).max())
    assert errs[2] < 1e-7 and errs[0] / errs[2] > 1e3
