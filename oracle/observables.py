"""Observables of Sec. II A on the grid.

<a|b> = dV * sum conj(a) b  (dV = product of grid spacings),
||psi|| = <psi|psi>^{1/2}, populations P_s = dV sum_j |psi_s(q_j)|^2,
E = <psi|H|psi>, symplectic form omega(psi, phi) = -2 hbar Im<psi|phi>
(Eq. def_symplectic_two_form).
"""
import numpy as np

HBAR = 1.0


def inner(a, b, dv):
    return dv * np.vdot(a.reshape(-1), b.reshape(-1))


def norm(psi, dv):
    return float(np.sqrt(inner(psi, psi, dv).real))


def populations(psi, dv):
    S = psi.shape[0]
    return np.array([dv * np.sum(np.abs(psi[s]) ** 2) for s in range(S)])


def energy(H, psi, dv):
    return float(inner(psi, (H @ psi.reshape(-1)).reshape(psi.shape), dv).real)


def omega(psi, phi, dv):
    return float(-2.0 * HBAR * inner(psi, phi, dv).imag)
