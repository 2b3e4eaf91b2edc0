"""Synthetic NaI-like two-state diabatic model (input data only).

The paper's NaI example uses a literature model whose functional form and
constants are not printed in the paper.  This module defines a stand-in of
the same character, labelled "NaI-like", NOT the literature model:

* covalent diabat  W_cc(q) = B exp(-q / rho_c)                (repulsive, -> 0)
* ionic diabat     W_ii(q) = E_ion - 1/q + A exp(-q / rho_i)   (Coulomb well)
* coupling         W_ci(q) = A_c exp(-beta_c (q - q_c)^2)

A and rho_i are fixed so that the ionic minimum sits at the printed Gaussian
centre q0 = 4.9889 a.u. with the curvature mu*omega^2 of a harmonic oscillator
whose ground state has the printed width sigma0 = 0.110436 a.u. (sigma0 read
as the standard deviation of |psi|^2, omega = 1 / (2 mu sigma0^2)), i.e. the
initial Gaussian is the harmonic ground state of the ground-state minimum, as
Sec. III describes.  E_ion, B, rho_c, A_c, beta_c, q_c are this project's
choices: the diabats cross near 13.1 a.u., the excited adiabatic state is
bound (Coulomb) and the ground adiabatic state dissociates, and a Landau-Zener
estimate gives a transfer of about 8 % -- qualitatively the behaviour
described for NaI in Sec. III.

Diabatic index 0 = covalent, 1 = ionic.  Arrays follow the library layout:
W has the S(S+1)/2 = 3 upper-triangle entries (00, 01, 11) per grid point,
dW their first derivatives with respect to q.
"""
import numpy as np

from .constants import NAI_REDUCED_MASS, NAI_Q0, NAI_SIGMA0, NAI_P0


def nai_like_params(mu=NAI_REDUCED_MASS, q0=NAI_Q0, sigma0=NAI_SIGMA0):
    """Constants of the NaI-like diabatic model (dict, Hartree atomic units)."""
    omega = 1.0 / (2.0 * mu * sigma0 ** 2)
    k = mu * omega ** 2
    # -1/q + A exp(-q/rho): zero slope and curvature k at q0
    rho_i = 1.0 / (q0 ** 2 * (k + 2.0 / q0 ** 3))
    a_ion = rho_i * np.exp(q0 / rho_i) / q0 ** 2
    rho_c = 1.5
    b_cov = 0.05 * np.exp(q0 / rho_c)     # covalent curve 0.05 Ha at q0
    return dict(E_ion=0.07644, A_ion=float(a_ion), rho_ion=float(rho_i),
                B_cov=float(b_cov), rho_cov=rho_c,
                A_c=0.002, beta_c=0.02, q_c=13.1, mu=mu, omega=omega)


def nai_like_diabatic(q, params=None):
    """Diabatic matrix and its derivative on the points q.

    Returns (W, dW) with W of shape (3, N) = (W00, W01, W11) and dW of shape
    (1, 3, N) (one nuclear dimension)."""
    p = params or nai_like_params()
    q = np.asarray(q, dtype=np.float64)
    e_c = p["B_cov"] * np.exp(-q / p["rho_cov"])
    w_cc = e_c
    d_cc = -e_c / p["rho_cov"]
    e_i = p["A_ion"] * np.exp(-q / p["rho_ion"])
    w_ii = p["E_ion"] - 1.0 / q + e_i
    d_ii = 1.0 / q ** 2 - e_i / p["rho_ion"]
    x = q - p["q_c"]
    w_ci = p["A_c"] * np.exp(-p["beta_c"] * x * x)
    d_ci = -2.0 * p["beta_c"] * x * w_ci
    W = np.stack([w_cc, w_ci, w_ii])
    dW = np.stack([d_cc, d_ci, d_ii])[None]
    return W, dW


def initial_gaussian_params(seed, q0=NAI_Q0, sigma0=NAI_SIGMA0, p0=NAI_P0):
    """Seeded centre, momentum and width of an initial Gaussian.

    seed None returns the printed values unchanged; otherwise
    q0 + 0.02 u and sigma0 (1 + 0.05 u') with u, u' ~ U(-1, 1) from PCG64."""
    if seed is None:
        return float(q0), float(p0), float(sigma0)
    u = np.random.default_rng(seed).uniform(-1.0, 1.0, 2)
    return float(q0 + 0.02 * u[0]), float(p0), float(sigma0 * (1.0 + 0.05 * u[1]))
