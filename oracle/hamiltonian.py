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
