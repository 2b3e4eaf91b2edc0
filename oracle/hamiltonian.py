"""Dense adiabatic molecular Hamiltonian, Eq. (adiab_mol_ham) (Sec. II E).

H = 1/2 [p 1 - i hbar F(q)]^dagger . m^{-1} . [p 1 - i hbar F(q)] + V(q)

with p_d = -i hbar D_d the momentum along dimension d (D_d the spectral
derivative), F a D-vector of real antisymmetric S x S coupling matrices and V
the diagonal adiabatic potential.  The operator is assembled literally as
sum_d (1/2 m_d) A_d^H A_d + V with A_d = p_d (x) 1_S - i hbar F_d, on the index
s * Ngrid + j (surface-major, grid points in C order).
"""
import numpy as np

from . import grid as _grid

HBAR = 1.0


def coupling_full(F_upper, S):
    """Expand the stored upper triangle F[d, pair, ...] (pairs (i<j) in
    lexicographic order) into full antisymmetric arrays Ff[d, i, j, ...]."""
    F_upper = np.asarray(F_upper, dtype=np.float64)
    D = F_upper.shape[0]
    gshape = F_upper.shape[2:]
    Ff = np.zeros((D, S, S) + gshape)
    pair = 0
    for i in range(S):
        for j in range(i + 1, S):
            Ff[:, i, j] = F_upper[:, pair]
            Ff[:, j, i] = -F_upper[:, pair]
            pair += 1
    return Ff


def dense_h(qmins, qmaxs, ns, mass, V, F_upper):
    """Dense (S*Ng) x (S*Ng) complex Hamiltonian.

    qmins, qmaxs, ns, mass: per-dimension lists; V: (S, *ns); F_upper:
    (D, S(S-1)/2, *ns)."""
    V = np.asarray(V, dtype=np.float64)
    S = V.shape[0]
    D = len(ns)
    ng = int(np.prod(ns))
    Ff = coupling_full(F_upper, S).reshape(D, S, S, ng)
    H = np.diag(V.reshape(S * ng).astype(np.complex128))
    for d in range(D):
        Dd = _grid.derivative_along(d, qmins, qmaxs, ns)
        p = -1j * HBAR * Dd
        A = np.kron(np.eye(S), p)
        for i in range(S):
            for j in range(S):
                if i != j:
                    A[i * ng:(i + 1) * ng, j * ng:(j + 1) * ng] += np.diag(-1j * HBAR * Ff[d, i, j])
        H += (A.conj().T @ A) / (2.0 * mass[d])
    return H


def apply_h(H, psi):
    """H psi for a state of shape (S, *grid)."""
    return (H @ psi.reshape(-1)).reshape(psi.shape)


def _derivative_kernel(qmin, qmax, n):
    """First column of the circulant D = Phi^{-1} diag(i k) Phi:
    d(m) = (1/n) sum_k i k_k exp(2 pi i k m / n), m = 0..n-1 (explicit sum)."""
    k = _grid.wavenumbers(qmin, qmax, n)
    d = np.empty(n, dtype=np.complex128)
    kk = np.arange(n)
    for m0 in range(0, n, 256):
        m = np.arange(m0, min(n, m0 + 256))
        ph = np.exp(2j * np.pi * ((np.outer(m, kk) % n) / n))
        d[m0:m0 + len(m)] = (ph @ (1j * k)) / n
    return d


def _circulant_apply(d, x, adjoint=False):
    """(D x)_j = sum_l d((j - l) mod n) x_l; adjoint: (D^H x)_j = sum_l conj(d((l - j) mod n)) x_l."""
    n = len(d)
    out = np.empty(n, dtype=np.complex128)
    l = np.arange(n)
    for j0 in range(0, n, 512):
        j = np.arange(j0, min(n, j0 + 512))
        if adjoint:
            blk = np.conj(d[(l[None, :] - j[:, None]) % n])
        else:
            blk = d[(j[:, None] - l[None, :]) % n]
        out[j0:j0 + len(j)] = blk @ x
    return out


def apply_h_matrix_free(qmin, qmax, n, mass, V, F_upper, psi):
    """H psi on a 1-D grid without forming H (for grids too large for dense
    matrices): A psi with A = p - i hbar F, p = -i hbar D, then
    H psi = (1/2m) A^H (A psi) + V psi with A^H = p^H + (-i hbar F)^H taken
    literally (conjugate transposes of the circulant D and of F)."""
    V = np.asarray(V, dtype=np.float64)
    S = V.shape[0]
    Ff = coupling_full(F_upper, S)[0]          # (S, S, n)
    d = _derivative_kernel(qmin, qmax, n)
    psi = np.asarray(psi, dtype=np.complex128).reshape(S, n)
    Apsi = np.empty_like(psi)
    for s in range(S):
        acc = -1j * HBAR * _circulant_apply(d, psi[s])
        for t in range(S):
            acc = acc - 1j * HBAR * Ff[s, t] * psi[t]
        Apsi[s] = acc
    out = np.empty_like(psi)
    for s in range(S):
        acc = np.conj(-1j * HBAR) * _circulant_apply(d, Apsi[s], adjoint=True)
        for t in range(S):
            acc = acc + np.conj(-1j * HBAR) * Ff[t, s] * Apsi[t]
        out[s] = acc / (2.0 * mass) + V[s] * psi[s]
    return out


def _circulant_along(d, x, axis, adjoint=False):
    """Apply the circulant derivative with first column d along one axis of x
    (explicit sums, line by line)."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    out = np.empty_like(x)
    flat_in = x.reshape(-1, x.shape[-1])
    flat_out = out.reshape(-1, x.shape[-1])
    for r in range(flat_in.shape[0]):
        flat_out[r] = _circulant_apply(d, flat_in[r], adjoint=adjoint)
    return np.moveaxis(out, -1, axis)


def apply_h_matrix_free_2d(qmins, qmaxs, ns, masses, V, F_upper, psi):
    """H psi on a 2-D grid without forming H:
    H = sum_d (1/2 m_d) A_d^H A_d + V,  A_d = p_d - i hbar F_d,  p_d = -i hbar D_d,
    D_d the circulant spectral derivative along axis d (explicit sums), the
    conjugate transposes taken literally.  V: (S, n0, n1); F_upper:
    (2, S(S-1)/2, n0, n1); psi: (S, n0, n1)."""
    V = np.asarray(V, dtype=np.float64)
    S = V.shape[0]
    Ff = coupling_full(F_upper, S)                # (2, S, S, n0, n1)
    psi = np.asarray(psi, dtype=np.complex128).reshape((S,) + tuple(ns))
    out = V * psi
    for ax in range(2):
        dker = _derivative_kernel(qmins[ax], qmaxs[ax], ns[ax])
        A = np.empty_like(psi)
        for s in range(S):
            acc = -1j * HBAR * _circulant_along(dker, psi[s], ax)
            for t in range(S):
                acc = acc - 1j * HBAR * Ff[ax, s, t] * psi[t]
            A[s] = acc
        for s in range(S):
            acc = np.conj(-1j * HBAR) * _circulant_along(dker, A[s], ax, adjoint=True)
            for t in range(S):
                acc = acc + np.conj(-1j * HBAR) * Ff[ax, t, s] * A[t]
            out[s] = out[s] + acc / (2.0 * masses[ax])
    return out
