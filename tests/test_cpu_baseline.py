"""The same-algorithm CPU baseline (oracle/cpu_baseline, FFT + Lanczos in C)
against the dense oracle: it is timed beside the GPU path, so it must compute
the same propagation."""
import numpy as np
import pytest

import workloads as wl
from oracle import cpu_baseline, fields, grid, hamiltonian as ham, initial, propagate as prop


@pytest.mark.parametrize("order", [2, 4, 8])
def test_cpu_baseline_matches_dense_oracle(order):
    qmin, qmax, n = 3.8, 12.0, 128
    q, dq = grid.points(qmin, qmax, n)
    W, dW = wl.nai_like_diabatic(q)
    V, F = fields.two_state(W, dW)
    H = ham.dense_h([qmin], [qmax], [n], [wl.NAI_REDUCED_MASS], V, F)
    psi0 = np.stack([initial.state_on_surface(2, 1, initial.gaussian([q], [q0], [p0], [0.35]))
                     for q0, p0 in ((5.2, 4.0), (6.0, -2.0), (5.5, 0.0))])
    dt = 25.0
    want = prop.DenseStepper(H).propagate_columns(psi0, dt, 2, prop.MIDPOINT, order, 1)
    got = psi0.copy()
    info = cpu_baseline.propagate(got, qmin, qmax, wl.NAI_REDUCED_MASS, V, F[0], order, dt, 2, tol=1e-15)
    assert info["status"] == 0 and info["threads"] >= 1 and info["hpsi"] > 0
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-11
