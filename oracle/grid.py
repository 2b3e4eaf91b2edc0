"""Fourier grid and the dynamic Fourier derivative as dense matrices (Sec. II D).

The derivative is the plain definition D = Phi^{-1} diag(i k) Phi, with the
explicit DFT matrix Phi_{jk} = exp(-2 pi i j k / N) and Phi^{-1} = Phi^H / N.
"""
import numpy as np


def points(qmin, qmax, n):
    """Grid points q_j = qmin + j dq, j = 0..n-1, dq = (qmax - qmin)/n."""
    dq = (qmax - qmin) / n
    return qmin + dq * np.arange(n, dtype=np.float64), dq


def wavenumbers(qmin, qmax, n):
    """k_j = 2 pi/(n dq) * (j for j < n/2, j - n otherwise); the Nyquist mode
    j = n/2 carries k = -pi/dq."""
    dq = (qmax - qmin) / n
    j = np.arange(n)
    m = np.where(j < n // 2, j, j - n).astype(np.float64)
    return 2.0 * np.pi / (n * dq) * m


def dft_matrix(n):
    """Phi_{jk} = exp(-2 pi i jk / n); jk reduced mod n in integers first."""
    jk = np.outer(np.arange(n), np.arange(n)) % n
    return np.exp(-2j * np.pi * jk / n)


def derivative_matrix(qmin, qmax, n):
    """Spectral first-derivative matrix D = Phi^{-1} diag(i k) Phi (n x n)."""
    phi = dft_matrix(n)
    k = wavenumbers(qmin, qmax, n)
    return (phi.conj().T / n) @ (1j * k[:, None] * phi)


def derivative_along(axis, qmins, qmaxs, ns):
    """Derivative along one axis of a D-dimensional grid, as a dense
    (prod n) x (prod n) matrix in C order (kron with identities)."""
    out = np.ones((1, 1), dtype=np.complex128)
    for d, n in enumerate(ns):
        m = derivative_matrix(qmins[d], qmaxs[d], n) if d == axis else np.eye(n)
        out = np.kron(out, m)
    return out
