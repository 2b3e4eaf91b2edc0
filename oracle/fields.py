"""Diabatic -> adiabatic fields (Sec. II E).

Two states, Eqs. (pot_diab2adiab), (..._orthogonal_transformation),
(nonadiab_c), evaluated literally in 50-significant-digit arithmetic so that
the cancellation in Delta = V_1 - W_11 (where W_12 is small) cannot spoil the
FP64 result:

  Wbar = (W11 + W22)/2, dW = W22 - W11, r = sqrt((dW/2)^2 + W12^2)
  V_{1,2} = Wbar +- r,  Delta = V_1 - W11,
  O = [[W12, -Delta], [Delta, W12]] / sqrt(W12^2 + Delta^2),
  F_12 = -F_21 = (W12' Delta - W12 Delta') / (W12^2 + Delta^2),
  Delta' = V_1' - W11',  V_1' = Wbar' + ((dW/2)(dW'/2) + W12 W12') / r.

The paper labels the upper surface 1 (V_1 = Wbar + r).  The library orders
surfaces by ascending energy, so the output is V[0] = V_2 (ground),
V[1] = V_1 (excited) and the stored coupling F[d, 0] = F_{ground,excited}
= F_21 = -F_12 (the same operator, relabelled).

general_adiabatic() is an independent route for any S: per-point symmetric
eigen-decomposition (LAPACK) and the Hellmann-Feynman identity
F_ij = <phi_i| W' |phi_j> / (V_j - V_i); it is used to pin two_state().
"""
import mpmath
import numpy as np

_DPS = 50


def _two_state_point(w11, w12, w22, d11, d12, d22):
    mp = mpmath.mp
    w11, w12, w22 = mp.mpf(w11), mp.mpf(w12), mp.mpf(w22)
    dW = w22 - w11
    wbar = (w11 + w22) / 2
    r = mp.sqrt((dW / 2) ** 2 + w12 ** 2)
    v1 = wbar + r
    v2 = wbar - r
    delta = v1 - w11
    out_f = []
    for (a11, a12, a22) in zip(d11, d12, d22):
        a11, a12, a22 = mp.mpf(a11), mp.mpf(a12), mp.mpf(a22)
        dWp = a22 - a11
        wbarp = (a11 + a22) / 2
        v1p = wbarp + ((dW / 2) * (dWp / 2) + w12 * a12) / r
        deltap = v1p - a11
        f12 = (a12 * delta - w12 * deltap) / (w12 ** 2 + delta ** 2)
        out_f.append(f12)
    return v1, v2, out_f


def two_state(W, dW):
    """Adiabatic V (2, *g) and stored coupling F (D, 1, *g) from the diabatic
    W (3, *g) = (W11, W12, W22) and dW (D, 3, *g) (derivative along each q_d)."""
    W = np.asarray(W, dtype=np.float64)
    dW = np.asarray(dW, dtype=np.float64)
    g = W.shape[1:]
    D = dW.shape[0]
    Wf = W.reshape(3, -1)
    dWf = dW.reshape(D, 3, -1)
    n = Wf.shape[1]
    V = np.empty((2, n))
    F = np.empty((D, 1, n))
    with mpmath.workdps(_DPS):
        for j in range(n):
            v1, v2, f12 = _two_state_point(Wf[0, j], Wf[1, j], Wf[2, j],
                                           dWf[:, 0, j], dWf[:, 1, j], dWf[:, 2, j])
            V[0, j] = float(v2)
            V[1, j] = float(v1)
            for d in range(D):
                F[d, 0, j] = -float(f12[d])
    return V.reshape((2,) + g), F.reshape((D, 1) + g)


def orthogonal_matrix(w11, w12, w22):
    """O(q) of Eq. (..._orthogonal_transformation) at one point (FP64), columns
    (upper, lower) in the paper's labelling."""
    dW = w22 - w11
    r = np.sqrt((dW / 2) ** 2 + w12 ** 2)
    delta = (w11 + w22) / 2 + r - w11
    nrm = np.sqrt(w12 ** 2 + delta ** 2)
    return np.array([[w12, -delta], [delta, w12]]) / nrm


def unpack_symmetric(Wu, S):
    """(S(S+1)/2, n) upper triangle (row-major pairs i<=j) -> (n, S, S)."""
    n = Wu.shape[-1]
    M = np.zeros((n, S, S))
    t = 0
    for i in range(S):
        for j in range(i, S):
            M[:, i, j] = Wu[t]
            M[:, j, i] = Wu[t]
            t += 1
    return M


def general_adiabatic(W, dW, S, gauge="continuity"):
    """Any S, 1-D grids: eigen-decomposition + Hellmann-Feynman.

    gauge "paper2" (S = 2 only) fixes the signs of Eq. (..._orthogonal_
    transformation) for W12 > 0 (upper eigenvector with positive first
    component, lower with positive second component); "continuity" makes the
    largest component of each eigenvector positive at the first point and
    keeps the overlap with the previous point positive."""
    W = np.asarray(W, dtype=np.float64)
    dW = np.asarray(dW, dtype=np.float64)
    D = dW.shape[0]
    n = W.shape[-1]
    M = unpack_symmetric(W.reshape(-1, n), S)
    Md = [unpack_symmetric(dW[d].reshape(-1, n), S) for d in range(D)]
    vals, vecs = np.linalg.eigh(M)          # ascending eigenvalues
    for j in range(n):
        for i in range(S):
            v = vecs[j, :, i]
            if gauge == "paper2":
                comp = 0 if i == 1 else 1
                if v[comp] < 0:
                    vecs[j, :, i] = -v
            else:
                if j == 0:
                    if v[np.argmax(np.abs(v))] < 0:
                        vecs[j, :, i] = -v
                elif np.dot(v, vecs[j - 1, :, i]) < 0:
                    vecs[j, :, i] = -v
    npair = S * (S - 1) // 2
    F = np.zeros((D, npair, n))
    for d in range(D):
        t = 0
        for i in range(S):
            for k in range(i + 1, S):
                num = np.einsum("ja,jab,jb->j", vecs[:, :, i], Md[d], vecs[:, :, k])
                F[d, t] = num / (vals[:, k] - vals[:, i])
                t += 1
    return vals.T.copy(), F, vecs
