"""Pins of the oracle's diabatic -> adiabatic transformation (Sec. II E)."""
import numpy as np

import workloads as wl
from oracle import fields, grid


def _nai(n=2048):
    q, dq = grid.points(wl.NAI_QMIN, wl.NAI_QMAX, n)
    W, dW = wl.nai_like_diabatic(q)
    return q, W, dW


def test_potentials_are_the_eigenvalues_of_W():
    q, W, dW = _nai()
    V, F = fields.two_state(W, dW)
    M = fields.unpack_symmetric(W, 2)
    ev = np.linalg.eigvalsh(M)
    np.testing.assert_allclose(V.T, ev, rtol=0, atol=1e-15)
    assert np.all(V[0] <= V[1])


def test_coupling_matches_hellmann_feynman():
    q, W, dW = _nai()
    V, F = fields.two_state(W, dW)
    V2, F2, _ = fields.general_adiabatic(W, dW, 2, gauge="paper2")
    np.testing.assert_allclose(F, F2, rtol=0, atol=1e-10 * np.abs(F).max())
    assert np.abs(F).max() > 0.1      # the avoided crossing is resolved


def test_coupling_is_the_derivative_of_the_orthogonal_matrix():
    # F = O^T O' (Sec. II E); stored F[0] = -F_12 of the paper's labelling
    q = np.linspace(11.5, 14.5, 41)
    h = 1e-5
    W, dW = wl.nai_like_diabatic(q)
    Wp, _ = wl.nai_like_diabatic(q + h)
    Wm, _ = wl.nai_like_diabatic(q - h)
    V, F = fields.two_state(W, dW)
    for j in range(len(q)):
        O = fields.orthogonal_matrix(W[0, j], W[1, j], W[2, j])
        Op = fields.orthogonal_matrix(Wp[0, j], Wp[1, j], Wp[2, j])
        Om = fields.orthogonal_matrix(Wm[0, j], Wm[1, j], Wm[2, j])
        Fp = O.T @ (Op - Om) / (2 * h)
        assert abs(Fp[0, 0]) < 1e-6 and abs(Fp[0, 1] + Fp[1, 0]) < 1e-6
        assert abs(-Fp[0, 1] - F[0, 0, j]) < 1e-6 * max(1.0, abs(F[0, 0, j]))


def test_orthogonal_matrix_diagonalises_W():
    q = np.linspace(10.0, 16.0, 13)
    W, dW = wl.nai_like_diabatic(q)
    V, F = fields.two_state(W, dW)
    for j in range(len(q)):
        O = fields.orthogonal_matrix(W[0, j], W[1, j], W[2, j])
        Wm = np.array([[W[0, j], W[1, j]], [W[1, j], W[2, j]]])
        Dg = O.T @ Wm @ O
        assert abs(Dg[0, 1]) < 1e-15
        assert abs(Dg[0, 0] - V[1, j]) < 1e-15 and abs(Dg[1, 1] - V[0, j]) < 1e-15


def test_nai_like_recipe_reproduces_printed_gaussian():
    # the ionic (ground-state) minimum is at q0 with harmonic width sigma0
    p = wl.nai_like_params()
    q = np.linspace(4.5, 5.5, 200001)
    W, dW = wl.nai_like_diabatic(q, p)
    j = np.argmin(W[2])
    assert abs(q[j] - wl.NAI_Q0) < 1e-4
    h = 1e-3
    Wp, _ = wl.nai_like_diabatic(np.array([wl.NAI_Q0 - h, wl.NAI_Q0, wl.NAI_Q0 + h]), p)
    k = (Wp[2, 0] - 2 * Wp[2, 1] + Wp[2, 2]) / h ** 2
    omega = np.sqrt(k / wl.NAI_REDUCED_MASS)
    sigma = np.sqrt(1.0 / (2 * wl.NAI_REDUCED_MASS * omega))
    assert abs(sigma - wl.NAI_SIGMA0) < 1e-6


def _three_state(q):
    # three displaced harmonic diabats with smooth positive couplings
    kf = 0.05
    w = [0.5 * kf * (q - 0.8) ** 2, 0.5 * kf * (q + 0.6) ** 2 + 0.01, 0.5 * kf * q ** 2 + 0.03]
    dw = [kf * (q - 0.8), kf * (q + 0.6), kf * q]
    cpl, dcpl = {}, {}
    for (a, b), (c, x0) in {(0, 1): (0.004, 0.1), (0, 2): (0.003, 1.0), (1, 2): (0.005, -0.8)}.items():
        g = c * np.exp(-(q - x0) ** 2 / 2.0) + 0.001
        cpl[(a, b)] = g
        dcpl[(a, b)] = -(q - x0) * (g - 0.001)
    W = np.stack([w[0], cpl[(0, 1)], cpl[(0, 2)], w[1], cpl[(1, 2)], w[2]])
    dW = np.stack([dw[0], dcpl[(0, 1)], dcpl[(0, 2)], dw[1], dcpl[(1, 2)], dw[2]])[None]
    return W, dW


def test_three_state_adiabatic_hamiltonian_has_the_diabatic_spectrum():
    from oracle import hamiltonian as ham
    qmin, qmax, n, m = -9.0, 9.0, 480, 400.0
    q, dq = grid.points(qmin, qmax, n)
    W, dW = _three_state(q)
    V, F, _ = fields.general_adiabatic(W, dW, 3)
    Ha = ham.dense_h([qmin], [qmax], [n], [m], V, F)
    D = grid.derivative_matrix(qmin, qmax, n)
    T = -(D @ D) / (2 * m)
    M = fields.unpack_symmetric(W, 3)
    Hd = np.kron(np.eye(3), T).astype(complex)
    for a in range(3):
        for b in range(3):
            Hd[a * n:(a + 1) * n, b * n:(b + 1) * n] += np.diag(M[:, a, b])
    ea = np.linalg.eigvalsh(Ha)[:20]
    ed = np.linalg.eigvalsh(Hd)[:20]
    np.testing.assert_allclose(ea, ed, rtol=0, atol=1e-9)


def test_three_state_coupling_is_the_derivative_of_the_eigenvectors():
    q = np.linspace(-3.0, 3.0, 30001)
    W, dW = _three_state(q)
    V, F, vecs = fields.general_adiabatic(W, dW, 3)
    h = q[1] - q[0]
    dvec = (vecs[2:] - vecs[:-2]) / (2 * h)
    t = 0
    for i in range(3):
        for k in range(i + 1, 3):
            fd = np.einsum("ja,ja->j", vecs[1:-1, :, i], dvec[:, :, k])
            assert np.abs(fd - F[0, t, 1:-1]).max() < 1e-4 * max(1.0, np.abs(F[0, t]).max())
            t += 1
