"""Gaussian initial state (Sec. III).

psi(q) = exp(-(q - q0)^2 / (4 sigma0^2) + i p0 (q - q0) / hbar), with sigma0
read as the standard deviation of |psi|^2, normalised on the grid so that
dq * sum_j |psi(q_j)|^2 = 1; in D dimensions the product of such factors.
"""
import numpy as np

HBAR = 1.0


def gaussian(qs, q0, p0, sigma0):
    """qs: list of 1-D point arrays (one per dimension); q0, p0, sigma0:
    per-dimension sequences.  Returns the normalised Gaussian on the grid."""
    psi = np.ones([len(q) for q in qs], dtype=np.complex128)
    dv = 1.0
    for d, q in enumerate(qs):
        x = q - q0[d]
        f = np.exp(-x * x / (4.0 * sigma0[d] ** 2) + 1j * p0[d] * x / HBAR)
        sh = [1] * len(qs)
        sh[d] = len(q)
        psi = psi * f.reshape(sh)
        dv *= q[1] - q[0]
    return psi / np.sqrt(dv * np.sum(np.abs(psi) ** 2))


def state_on_surface(S, surface, psi_grid):
    """Molecular state (S, *grid) with psi_grid on one surface, zero elsewhere."""
    out = np.zeros((S,) + psi_grid.shape, dtype=np.complex128)
    out[surface] = psi_grid
    return out
