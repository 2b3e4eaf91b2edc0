"""Pins of the oracle's elementary comparison methods (Sec. II B,
Appendix A): explicit and implicit Euler (Eqs. exp_euler, imp_euler) and
second-order differencing (Eq. sod_method) with its Runge-Kutta start.

* norm identities of the Euler methods (Eqs. exp_eu_norm, imp_eu_norm, here
  exact because the steps are applied exactly):
  ||(1 - i e H) psi||^2 = ||psi||^2 + e^2 <H^2>_psi and
  ||psi||^2 = ||psi'||^2 + e^2 <H^2>_psi' for psi' = (1 + i e H)^{-1} psi;
* global order 1 (Euler) and 2 (SOD) against e^{-iHt} -- a wrong sign of i
  gives order 0 and fails;
* Proposition 4 and Eq. sod_energy_a: (<psi(t)|phi(t - e)> + <psi(t - e)|phi(t)>)/2
  and Re<psi(t)|H|psi(t + e)> are conserved exactly along a SOD run;
* stability: SOD stays bounded for e < 1/E_max and diverges beyond it
  (Eq. sod_critical_timestep);
* the two-stage Runge-Kutta start has local error O(e^3).
"""
import numpy as np
import pytest

from oracle import propagate as prop


@pytest.fixture(scope="module")
def herm():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    H = (A + A.conj().T) / 8.0
    psi = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    phi = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    return H, psi / np.linalg.norm(psi), phi / np.linalg.norm(phi)


def _h2(H, v):
    return float(np.vdot(H @ v, H @ v).real)


def test_euler_norm_identities(herm):
    H, psi, _ = herm
    st = prop.DenseStepper(H)
    e = 0.37
    a = st.expl(psi, e)
    assert abs(np.vdot(a, a).real - (1.0 + e * e * _h2(H, psi))) < 1e-13
    b = st.impl(psi, e)
    assert abs(1.0 - (np.vdot(b, b).real + e * e * _h2(H, b))) < 1e-13
    # many steps: explicit Euler grows the norm, implicit Euler shrinks it
    assert np.linalg.norm(st.euler_steps(psi, e, 50, prop.EXPLICIT_EULER)) > 1.5
    assert np.linalg.norm(st.euler_steps(psi, e, 50, prop.IMPLICIT_EULER)) < 0.7


@pytest.mark.parametrize("method,order", [(prop.EXPLICIT_EULER, 1), (prop.IMPLICIT_EULER, 1), (prop.SOD, 2)])
def test_global_order(herm, method, order):
    H, psi, _ = herm
    st = prop.DenseStepper(H)
    t = 2.0
    ex = prop.exact(H, psi, t)
    err = []
    for n in (200, 400):
        if method == prop.SOD:
            got = st.sod(psi, t / n, n)[0]
        else:
            got = st.euler_steps(psi, t / n, n, method)
        err.append(np.linalg.norm(got - ex))
    slope = np.log(err[0] / err[1]) / np.log(2.0)
    assert abs(slope - order) < 0.15, (err, slope)


def test_rk2_start_local_order(herm):
    H, psi, _ = herm
    st = prop.DenseStepper(H)
    err = [np.linalg.norm(st.rk2(psi, -h) - prop.exact(H, psi, -h)) for h in (0.02, 0.01)]
    assert abs(np.log(err[0] / err[1]) / np.log(2.0) - 3.0) < 0.1


def test_sod_conserved_quantities(herm):
    H, psi, phi = herm
    st = prop.DenseStepper(H)
    e = 0.3
    ps_cur, ps_prev = st.sod(psi, e, 0)
    ph_cur, ph_prev = st.sod(phi, e, 0)
    inner0 = 0.5 * (np.vdot(ps_cur, ph_prev) + np.vdot(ps_prev, ph_cur))
    norm0 = np.vdot(ps_cur, ps_prev).real
    ps_next = st.sod(ps_cur, e, 1, psi_prev=ps_prev)[0]
    en0 = np.vdot(ps_cur, H @ ps_next).real
    for _ in range(5):
        ps_cur, ps_prev = st.sod(ps_cur, e, 37, psi_prev=ps_prev)
        ph_cur, ph_prev = st.sod(ph_cur, e, 37, psi_prev=ph_prev)
        inner = 0.5 * (np.vdot(ps_cur, ph_prev) + np.vdot(ps_prev, ph_cur))
        assert abs(inner - inner0) < 1e-13
        assert abs(np.vdot(ps_cur, ps_prev).real - norm0) < 1e-13
        ps_next = st.sod(ps_cur, e, 1, psi_prev=ps_prev)[0]
        assert abs(np.vdot(ps_cur, H @ ps_next).real - en0) < 1e-13
    # the true norm is only conserved to O(e^2) per run, not exactly
    assert abs(np.linalg.norm(ps_cur) - 1.0) > 1e-8


def test_sod_stability_limit(herm):
    H, psi, _ = herm
    st = prop.DenseStepper(H)
    emax = np.abs(np.linalg.eigvalsh(H)).max()
    stable = st.sod(psi, 0.95 / emax, 3000)[0]
    assert np.linalg.norm(stable) < 20.0
    unstable = st.sod(psi, 1.05 / emax, 200)[0]
    assert np.linalg.norm(unstable) > 1e6
