"""Two-dimensional two-state model (input data only): an avoided-crossing
mode q1 linearly coupled to a harmonic spectator mode q2.

  W11 = k1 (q1 - a)^2 / 2 + k2 q2^2 / 2 + kappa q2
  W22 = k1 (q1 + a)^2 / 2 + k2 q2^2 / 2 + delta0 - kappa q2
  W12 = c  (> 0 everywhere: no conical intersection, finite couplings)

The spectator mode tunes the diabatic gap linearly.  The initial Gaussian
sits on the excited adiabatic surface at the minimum of W11 (vertical
excitation), with the harmonic ground-state widths of that well.
"""
import numpy as np

PARAMS = dict(k1=0.02, a=0.8, k2=0.05, kappa=0.01, delta0=0.005, c=0.004, mass=(5000.0, 5000.0),
              qmin=(-4.5, -3.0), qmax=(4.5, 3.0))


def model2d_diabatic(q1, q2, p=None):
    """W (3, n0, n1) = (W11, W12, W22) on the product grid and dW (2, 3, n0, n1)."""
    p = p or PARAMS
    Q1, Q2 = np.meshgrid(np.asarray(q1, float), np.asarray(q2, float), indexing="ij")
    w11 = 0.5 * p["k1"] * (Q1 - p["a"]) ** 2 + 0.5 * p["k2"] * Q2 ** 2 + p["kappa"] * Q2
    w22 = 0.5 * p["k1"] * (Q1 + p["a"]) ** 2 + 0.5 * p["k2"] * Q2 ** 2 + p["delta0"] - p["kappa"] * Q2
    w12 = np.full_like(Q1, p["c"])
    d1 = np.stack([p["k1"] * (Q1 - p["a"]), np.zeros_like(Q1), p["k1"] * (Q1 + p["a"])])
    d2 = np.stack([p["k2"] * Q2 + p["kappa"], np.zeros_like(Q1), p["k2"] * Q2 - p["kappa"]])
    W = np.ascontiguousarray(np.stack([w11, w12, w22]))
    dW = np.ascontiguousarray(np.stack([d1, d2]))
    return W, dW


def model2d_initial(p=None):
    """(q0, p0, sigma0) per dimension for the Gaussian on the excited surface."""
    p = p or PARAMS
    m1, m2 = p["mass"]
    w1 = np.sqrt(p["k1"] / m1)
    w2 = np.sqrt(p["k2"] / m2)
    return [p["a"], 0.0], [0.0, 0.0], [float(np.sqrt(1 / (2 * m1 * w1))), float(np.sqrt(1 / (2 * m2 * w2)))]
