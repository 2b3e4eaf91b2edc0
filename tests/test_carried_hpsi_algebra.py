"""The algebra behind carrying H psi (and H^2 psi) across implicit-midpoint
sub-steps, checked with the oracle's exact solves: for (1 + i tau H) chi =
psi, H chi = i (chi - psi) / tau and H^2 chi = i (H chi - H psi) / tau, so
for psi' = 2 chi - psi the recurrences H psi' = 2 H chi - H psi and
H^2 psi' = 2 H^2 chi - H^2 psi reproduce the directly applied operator
along a whole composed step, with the error changing sign each sub-step
instead of growing."""
import numpy as np

import workloads as wl
from oracle import composition as comp, fields, grid, hamiltonian as ham, initial, propagate as prop


def test_carried_h_psi_matches_direct_application():
    qmin, qmax, n = 3.8, 12.0, 64
    q, dq = grid.points(qmin, qmax, n)
    W, dW = wl.nai_like_diabatic(q)
    V, F = fields.two_state(W, dW)
    H = ham.dense_h([qmin], [qmax], [n], [wl.NAI_REDUCED_MASS], V, F)
    st = prop.DenseStepper(H)
    psi = initial.state_on_surface(2, 1, initial.gaussian([q], [5.5], [2.0], [0.4])).reshape(-1)
    dt = 20.0
    hp = H @ psi                  # exact at the start of the composed step
    h2 = H @ hp
    worst1 = worst2 = 0.0
    for f in comp.schedule(8, comp.SUZUKI):
        tau = 0.5 * f * dt
        chi = st.impl(psi, tau).reshape(-1)
        hchi = 1j * (chi - psi) / tau
        h2chi = 1j * (hchi - hp) / tau
        psi = 2 * chi - psi
        hp = 2 * hchi - hp
        h2 = 2 * h2chi - h2
        worst1 = max(worst1, np.linalg.norm(hp - H @ psi) / np.linalg.norm(H @ psi))
        worst2 = max(worst2, np.linalg.norm(h2 - H @ (H @ psi)) / np.linalg.norm(H @ (H @ psi)))
    # 125 sub-steps of Suzuki order 8 (|tau| up to 1.4 a.u.): the carried
    # values stay within rounding of the directly applied operator (about
    # 5e-13 for H psi, 7e-10 for H^2 psi, which is divided by tau twice)
    assert worst1 < 1e-11
    assert worst2 < 1e-8
