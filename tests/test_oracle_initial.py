"""Pins of the Gaussian initial state (Sec. III) and of the printed numbers."""
import json
import os

import numpy as np

import workloads as wl
from oracle import grid, initial

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_workload_constants_are_the_printed_values():
    g = GOLD["nai_grid"]
    assert (wl.NAI_N, wl.NAI_QMIN, wl.NAI_QMAX) == (g["N"], g["qmin"], g["qmax"])
    p = GOLD["nai_initial_gaussian"]
    assert (wl.NAI_Q0, wl.NAI_P0, wl.NAI_SIGMA0) == (p["q0"], p["p0"], p["sigma0"])
    assert wl.NAI_TF == GOLD["nai_final_time"]["t_f"]
    assert (wl.PHI_Q0, wl.PHI_P0) == (GOLD["second_gaussian_phi"]["q0"], GOLD["second_gaussian_phi"]["p0"])


def test_gaussian_moments():
    # sigma0 is the standard deviation of |psi|^2; minimum uncertainty in p
    qmin, qmax, n = 3.8, 47.0, 2048
    q, dq = grid.points(qmin, qmax, n)
    q0, p0, s0 = wl.PHI_Q0, wl.PHI_P0, wl.NAI_SIGMA0
    psi = initial.gaussian([q], [q0], [p0], [s0])
    rho = np.abs(psi) ** 2 * dq
    assert abs(rho.sum() - 1.0) < 1e-14
    mean = (rho * q).sum()
    var = (rho * (q - mean) ** 2).sum()
    assert abs(mean - q0) < 1e-12 and abs(np.sqrt(var) - s0) < 1e-10
    D = grid.derivative_matrix(qmin, qmax, n)
    dpsi = D @ psi
    pm = (np.vdot(psi, -1j * dpsi) * dq).real
    p2 = (np.vdot(dpsi, dpsi) * dq).real
    assert abs(pm - p0) < 1e-10
    assert abs(np.sqrt(p2 - pm ** 2) - 1.0 / (2 * s0)) < 1e-8
