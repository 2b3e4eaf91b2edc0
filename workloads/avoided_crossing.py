"""Seeded one-dimensional avoided-crossing models for the batched workload
(input data only: diabatic matrices, their derivatives and Gaussian
parameters; the adiabatic fields are computed by the library and the oracle).

Model i (seed = base + i):
  S ~ U{2, 3}; N = 2^U{8..13}; grid q in [0, L), L = N * 0.025 a.u.;
  diabats W_kk(q) = s_k a tanh((q - c_k)/a) + o_k + wall(q): linear with
  slope s_k near c_k (|s_k| ~ U(0.01, 0.05) Ha/a.u., alternating sign),
  saturating over a = 8 a.u. so the energy range stays below about 1 Ha on
  every box; wall(q) = 0.05 (exp(-(q - 1.15)/0.5) + exp((q - L + 1.15)/0.5))
  Ha is common to all states (0.5 Ha at the edges);
  states 0 and 1 cross at c_0 = c_1 = q_c ~ U(0.3, 0.7) L; for S = 3 the
  third diabat crosses diabat 1 at c_2 ~ U(0.3, 0.7) L;
  couplings W_kl(q) = (g_kl / 2) exp(-(q - x_kl)^2 / (2 w_kl^2)) centred at the
  grid crossing x_kl of diabats k and l (the box centre if they do not
  cross), gap g_kl ~ U(1e-3, 2e-2) Ha, width w_kl ~ U(0.2, 2) a.u.;
  mass: the NaI reduced mass; psi0: Gaussian on the top adiabatic surface at
  q0 = 0.12 L + 1, p0 = 0, sigma0 = 0.3 a.u.
"""
import numpy as np

from .constants import NAI_REDUCED_MASS

DQ = 0.025
SAT = 8.0


def avoided_crossing_model(seed):
    rng = np.random.default_rng(seed)
    S = int(rng.integers(2, 4))
    N = int(2 ** rng.integers(8, 14))
    L = N * DQ
    q = DQ * np.arange(N)
    e1 = np.exp(-(q - 1.15) / 0.5)
    e2 = np.exp((q - L + 1.15) / 0.5)
    wall = 0.05 * (e1 + e2)
    dwall = 0.05 * (-e1 + e2) / 0.5
    qc = rng.uniform(0.3, 0.7) * L
    s = [rng.uniform(0.01, 0.05), -rng.uniform(0.01, 0.05), rng.uniform(0.01, 0.05)]
    c = [qc, qc, rng.uniform(0.3, 0.7) * L]
    o = [0.0, 0.0, 0.0]
    if S == 3:
        s[2] = s[0] * rng.uniform(0.3, 0.7)
        o[2] = s[1] * SAT * np.tanh((c[2] - qc) / SAT)
    diag = [s[k] * SAT * np.tanh((q - c[k]) / SAT) + o[k] + wall for k in range(S)]
    ddiag = [s[k] / np.cosh((q - c[k]) / SAT) ** 2 + dwall for k in range(S)]

    def crossing(k, l):
        d = diag[k] - diag[l]
        idx = np.nonzero(np.sign(d[1:]) != np.sign(d[:-1]))[0]
        if len(idx) == 0:
            return 0.5 * L
        j = idx[np.argmin(np.abs(idx - N // 2))]
        return float(q[j] + DQ * d[j] / (d[j] - d[j + 1]))

    W, dW = [], []
    for k in range(S):
        for l in range(k, S):
            if k == l:
                W.append(diag[k])
                dW.append(ddiag[k])
            else:
                g = rng.uniform(1e-3, 2e-2)
                w = rng.uniform(0.2, 2.0)
                x0 = crossing(k, l)
                cpl = 0.5 * g * np.exp(-(q - x0) ** 2 / (2 * w * w))
                W.append(cpl)
                dW.append(-(q - x0) / (w * w) * cpl)
    return dict(seed=seed, S=S, N=N, qmin=0.0, qmax=L, mass=NAI_REDUCED_MASS,
                W=np.ascontiguousarray(np.stack(W)), dW=np.ascontiguousarray(np.stack(dW)[None]),
                q0=0.12 * L + 1.0, p0=0.0, sigma0=0.3, surface=S - 1)
