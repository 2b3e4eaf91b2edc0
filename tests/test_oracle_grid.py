"""Pins of the oracle's Fourier grid (dynamic Fourier method, Sec. II D)."""
import numpy as np

from oracle import grid


def test_dft_matrix_is_the_library_fft():
    rng = np.random.default_rng(1)
    for n in (8, 16, 64, 128):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        np.testing.assert_allclose(grid.dft_matrix(n) @ x, np.fft.fft(x), rtol=0, atol=1e-11 * n)


def test_wavenumber_convention():
    qmin, qmax, n = 3.8, 47.0, 2048
    k = grid.wavenumbers(qmin, qmax, n)
    L = qmax - qmin
    dq = L / n
    assert np.isclose(k[1], 2 * np.pi / L) and np.isclose(k[-1], -2 * np.pi / L)
    assert np.isclose(k[n // 2], -np.pi / dq)
    assert k[0] == 0.0


def test_derivative_exact_on_every_grid_plane_wave():
    # D e^{i k q} = i k e^{i k q} exactly for every grid wave number, Nyquist included
    qmin, qmax, n = -3.0, 5.0, 32
    q, dq = grid.points(qmin, qmax, n)
    k = grid.wavenumbers(qmin, qmax, n)
    D = grid.derivative_matrix(qmin, qmax, n)
    for j in range(n):
        f = np.exp(1j * k[j] * q)
        np.testing.assert_allclose(D @ f, 1j * k[j] * f, rtol=0, atol=1e-11 * np.abs(k).max())


def test_derivative_spectral_accuracy_on_gaussian():
    qmin, qmax, n = -10.0, 10.0, 128
    q, dq = grid.points(qmin, qmax, n)
    f = np.exp(-q ** 2)
    D = grid.derivative_matrix(qmin, qmax, n)
    np.testing.assert_allclose((D @ f).real, -2 * q * f, rtol=0, atol=1e-12)
    assert np.abs((D @ f).imag).max() < 1e-12


def test_derivative_is_antihermitian():
    D = grid.derivative_matrix(0.0, 7.0, 64)
    assert np.abs(D + D.conj().T).max() < 1e-12


def test_derivative_along_axis_of_separable_function():
    qm, qx, ns = [-9.0, -10.0], [9.0, 10.0], [48, 56]
    q1, _ = grid.points(qm[0], qx[0], ns[0])
    q2, _ = grid.points(qm[1], qx[1], ns[1])
    g = np.exp(-q1 ** 2 / 2)
    h = np.exp(-q2 ** 2 / 3)
    f = np.outer(g, h).reshape(-1)
    D1 = grid.derivative_along(0, qm, qx, ns)
    D2 = grid.derivative_along(1, qm, qx, ns)
    np.testing.assert_allclose((D1 @ f).real, np.outer(-q1 * g, h).reshape(-1), atol=1e-7)
    np.testing.assert_allclose((D2 @ f).real, np.outer(g, -2 * q2 / 3 * h).reshape(-1), atol=1e-7)
