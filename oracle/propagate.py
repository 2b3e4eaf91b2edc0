"""Elementary and composed integrators with dense linear algebra (Sec. II B-C).

U_expl(e)  = 1 - i e H / hbar                           Eq. (exp_euler)
U_impl(e)  = (1 + i e H / hbar)^{-1}                    Eq. (imp_euler)
SOD        psi(t+e) = psi(t-e) - 2 i e H psi(t) / hbar  Eq. (sod_method)
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
EXPLICIT_EULER = 2
IMPLICIT_EULER = 3
SOD = 4


class DenseStepper:
    def __init__(self, H):
        self.H = np.asarray(H, dtype=np.complex128)
        self.n = self.H.shape[0]
        self._lu = {}

    def expl(self, psi, eps):
        v = psi.reshape(-1)
        return (v - 1j * eps / HBAR * (self.H @ v)).reshape(psi.shape)

    def _solve(self, rhs, eps):
        """(1 + i eps H / hbar)^{-1} rhs; rhs a vector or an (n, k) matrix."""
        key = float(eps)
        if key not in self._lu:
            A = np.eye(self.n, dtype=np.complex128) + 1j * eps / HBAR * self.H
            self._lu[key] = sla.lu_factor(A, check_finite=False)
        return sla.lu_solve(self._lu[key], rhs, check_finite=False)

    def impl(self, psi, eps):
        return self._solve(psi.reshape(-1), eps).reshape(psi.shape)

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

    def propagate_columns(self, states, dt, nsteps, method, order=2, scheme=composition.SUZUKI):
        """The same composed steps applied to several states at once: states
        is a sequence of k states (or an (k, ...) array); every implicit
        Euler factor is one LU solve with k right-hand sides.  Returns an
        array of the k propagated states."""
        states = np.asarray(states, dtype=np.complex128)
        shape = states.shape
        P = states.reshape(shape[0], self.n).T.copy()
        fr = composition.schedule(order, scheme)
        for _ in range(nsteps):
            for f in fr:
                eps = f * dt / 2
                if method == TRAPEZOIDAL:
                    P = self._solve(P - 1j * eps / HBAR * (self.H @ P), eps)
                elif method == MIDPOINT:
                    X = self._solve(P, eps)
                    P = X - 1j * eps / HBAR * (self.H @ X)
                else:
                    raise ValueError("unknown method %r" % (method,))
        return P.T.reshape(shape)


    def euler_steps(self, psi, eps, nsteps, method):
        """nsteps explicit (Eq. exp_euler) or implicit (Eq. imp_euler) Euler
        steps of size eps: first order, neither unitary nor symmetric."""
        for _ in range(nsteps):
            if method == EXPLICIT_EULER:
                psi = self.expl(psi, eps)
            elif method == IMPLICIT_EULER:
                psi = self.impl(psi, eps)
            else:
                raise ValueError("unknown Euler method %r" % (method,))
        return psi

    def rk2(self, psi, h):
        """One two-stage Runge-Kutta step of size h (h < 0 steps backward) of
        d psi/dt = -(i/hbar) H psi: k1 = f(psi), k2 = f(psi + h k1 / 2),
        psi + h k2."""
        v = psi.reshape(-1)
        k1 = -1j / HBAR * (self.H @ v)
        k2 = -1j / HBAR * (self.H @ (v + 0.5 * h * k1))
        return (v + h * k2).reshape(psi.shape)

    def sod(self, psi, eps, nsteps, psi_prev=None):
        """Second-order differencing, Eq. (sod_method):
        psi(t + eps) = psi(t - eps) - 2 (i/hbar) eps H psi(t).
        The missing psi(-eps) is approximated by one two-stage Runge-Kutta
        step backward from psi(0) (Sec. III), unless given.  Returns
        (psi(n eps), psi((n - 1) eps))."""
        prev = self.rk2(psi, -eps) if psi_prev is None else psi_prev
        cur = psi
        for _ in range(nsteps):
            nxt = (prev.reshape(-1) - 2j * eps / HBAR * (self.H @ cur.reshape(-1))).reshape(psi.shape)
            prev, cur = cur, nxt
        return cur, prev


def exact(H, psi, t):
    """e^{-iHt/hbar} psi through the Hermitian eigen-decomposition (LAPACK)."""
    lam, U = np.linalg.eigh(H)
    c = U.conj().T @ psi.reshape(-1)
    return (U @ (np.exp(-1j * lam * t / HBAR) * c)).reshape(psi.shape)


class ExactEvolution:
    """e^{-iHt/hbar} for many states and times from one Hermitian
    eigen-decomposition of H (the same definition as exact())."""

    def __init__(self, H):
        self.lam, self.U = np.linalg.eigh(np.asarray(H, dtype=np.complex128))

    def __call__(self, psi, t):
        c = self.U.conj().T @ psi.reshape(-1)
        return (self.U @ (np.exp(-1j * self.lam * t / HBAR) * c)).reshape(psi.shape)


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
