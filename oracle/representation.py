"""The diabatic representation and changes of grid (Sec. II E, Appendix B).

* diabatic_h: H_diab = (1/2) p^T m^{-1} p 1 + W(q) on the grid, with
  p = -i hbar D (D the spectral derivative, Sec. II D), so its kinetic part is
  -(hbar^2/2m) D^2 on every surface, and W(q) the real symmetric diabatic
  matrix at each point (no vector coupling).
* to_adiabatic / to_diabatic: psi = O(q)^T psi_diab (Eq. psi_diab2adiab),
  O(q) the orthogonal matrix of Eq. (pot_diab2adiab_orthogonal_transformation)
  for S = 2 (columns: the adiabatic states; the library order is ascending,
  so column 0 is the paper's lower state 2 and column 1 the upper state 1),
  or the eigenvectors of general_adiabatic for any S.
* trig_interpolate: the trigonometric interpolant of a periodic grid function
  (Appendix B compares wavepackets on grids of different density this way),
  p(q) = (1/N) sum_k c_k exp(i k (q - qmin)) with c = DFT of the samples and
  the Nyquist coefficient split evenly between +k and -k (a cosine), so that
  a real grid function has a real interpolant.  Points outside
  [qmin, qmax) see the periodic extension.
"""
import numpy as np

from . import fields, grid as _grid, hamiltonian as _ham

HBAR = 1.0


def diabatic_h(qmin, qmax, n, mass, W_upper, S):
    """Dense (S n) x (S n) diabatic Hamiltonian, 1-D grid; W_upper holds the
    S(S+1)/2 upper-triangle rows (00, 01, ..., 11, ...) of n values."""
    D = _grid.derivative_matrix(qmin, qmax, n)
    p = -1j * HBAR * D
    T = (p.conj().T @ p) / (2.0 * mass)
    H = np.kron(np.eye(S), T).astype(np.complex128)
    Wm = fields.unpack_symmetric(np.asarray(W_upper, dtype=np.float64).reshape(-1, n), S)   # (n, S, S)
    for a in range(S):
        for b in range(S):
            H[a * n:(a + 1) * n, b * n:(b + 1) * n] += np.diag(Wm[:, a, b])
    return H


def rotation(W_upper, S, dW=None):
    """O(q) at every point, shape (n, S, S), columns = adiabatic states in
    ascending energy.  S = 2: the paper's closed form (columns reordered to
    ascending); S > 2: the eigenvectors of general_adiabatic (needs dW)."""
    W_upper = np.asarray(W_upper, dtype=np.float64)
    n = W_upper.shape[-1]
    if S == 2:
        O = np.empty((n, 2, 2))
        for j in range(n):
            Op = fields.orthogonal_matrix(W_upper[0, j], W_upper[1, j], W_upper[2, j])   # (upper, lower)
            O[j, :, 0] = Op[:, 1]
            O[j, :, 1] = Op[:, 0]
        return O
    _, _, vecs = fields.general_adiabatic(W_upper, dW, S)
    return vecs


def to_adiabatic(O, psi_diab):
    """psi = O^T psi_diab at every point (psi arrays of shape (S, n))."""
    return np.einsum("jrs,rj->sj", O, psi_diab)


def to_diabatic(O, psi_adiab):
    """psi_diab = O psi (the inverse: O is orthogonal)."""
    return np.einsum("jrs,sj->rj", O, psi_adiab)


def trig_interpolate(values, qmin, qmax, q_out):
    """Trigonometric interpolant of the samples `values` (last axis: n points
    on [qmin, qmax)) evaluated at q_out, by explicit sums."""
    values = np.asarray(values, dtype=np.complex128)
    n = values.shape[-1]
    L = qmax - qmin
    j = np.arange(n)
    m = np.where(j < n // 2, j, j - n)
    c = values @ np.exp(-2j * np.pi * np.outer(j, m) / n)     # c_m = sum_j v_j e^{-2 pi i j m / n}
    x = (np.asarray(q_out, dtype=np.float64) - qmin) / L
    E = np.exp(2j * np.pi * np.outer(m, x))                  # (n, n_out)
    nyq = n // 2
    E[nyq] = np.cos(2 * np.pi * nyq * x)                     # -n/2 and +n/2 halves together
    return (c @ E) / n


def adiabatic_h_from_diabatic(qmin, qmax, n, mass, W_upper, dW):
    """Dense adiabatic H (Eq. adiab_mol_ham) of a two-state diabatic model."""
    V, F = fields.two_state(W_upper, dW)
    return _ham.dense_h([qmin], [qmax], [n], [mass], V, F)
