"""Elementary and composed integrators with dense linear algebra (Sec. II B-C).

U_expl(e)  = 1 - i e H / hbar                           Eq. (exp_euler)
U_impl(e)  = (1 + i e H / hbar)^{-1}                    Eq. (imp_euler)
U_trap(dt) = U_impl(dt/2) U_expl(dt/2)                  Eq. (trap_rule)
U_midp(dt) = U_expl(dt/2) U_impl(dt/2)                  Eq. (imp_midpoint)
composed   = product over the flat schedule of composition.schedule().

The implicit Euler factor is a dense complex LU with partial pivoting
(LAPACK), factored once per distinct step and cached.  exact() and
cayley_by_eigen() are the independent eigen-decomposition routes used to pin
the LU route.
"""
import numpy as np
import scipy.linalg as sla

from . import composition

HBAR = 1.0
TRAPEZOIDAL = 0
MIDPOINT = 1


class DenseStepper:
    def __init__(self, H):
        self.H = np.asarray(H, dtype=np.complex128)
        self.n = self.H.shape[0]
        self._lu = {}

    def expl(self, psi, eps):
        v = psi.reshape(-1)
        return (v - 1j * eps / HBAR * (self.H @ v)).reshape(psi.shape)

    def impl(self, psi, eps):
        key = float(eps)
        if key not in self._lu:
            A = np.eye(self.n, dtype=np.complex128) + 1j * eps / HBAR * self.H
            self._lu[key] = sla.lu_factor(A, check_finite=False)
        x = sla.lu_solve(self._lu[key], psi.reshape(-1), check_finite=False)
        return x.reshape(psi.shape)

    def trap(self, psi, dt):
        return self.impl(self.expl(psi, dt / 2), dt / 2)

    def midpoint(self, psi, dt):
        return self.expl(self.impl(psi, dt / 2), dt / 2)

    def elementary(self, psi, dt, method):
        if method == TRAPEZOIDAL:
            return self.trap(psi, dt)
        if method == MIDPOINT:
            return self.midpoint(psi, dt)
        raise ValueError("unknown method %r" % (method,))

    def composed(self, psi, dt, method, order, scheme):
        for f in composition.schedule(order, scheme):
            psi = self.elementary(psi, f * dt, method)
        return psi

    def propagate(self, psi, dt, nsteps, method, order=2, scheme=composition.SUZUKI):
        for _ in range(nsteps):
            psi = self.composed(psi, dt, method, order, scheme)
        return psi


def exact(H, psi, t):
    """e^{-iHt/hbar} psi through the Hermitian eigen-decomposition (LAPACK)."""
    lam, U = np.linalg.eigh(H)
    c = U.conj().T @ psi.reshape(-1)
    return (U @ (np.exp(-1j * lam * t / HBAR) * c)).reshape(psi.shape)


def cayley_by_eigen(H, psi, dt, fractions, nsteps=1):
    """Composed Cayley steps through the eigen-decomposition: every elementary
    step multiplies eigen-component lambda by R(f dt lambda / hbar) with
    R(x) = (1 - i x/2) / (1 + i x/2)."""
    lam, U = np.linalg.eigh(H)
    c = U.conj().T @ psi.reshape(-1)
    g = np.ones_like(lam, dtype=np.complex128)
    for f in fractions:
        x = f * dt * lam / HBAR
        g = g * (1 - 0.5j * x) / (1 + 0.5j * x)
    return (U @ (g ** nsteps * c)).reshape(psi.shape)
