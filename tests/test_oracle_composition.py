"""Pins of the composition schemes (Sec. II C) and the elementary Cayley step."""
import json
import os

import numpy as np
import pytest

from oracle import composition as comp, propagate as prop

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("scheme", [comp.TRIPLE_JUMP, comp.SUZUKI])
@pytest.mark.parametrize("p", [2, 4, 6])
def test_coefficients_sum_palindrome_and_order_condition(scheme, p):
    g = np.array(comp.gammas(scheme, p))
    assert abs(g.sum() - 1.0) < 1e-15
    np.testing.assert_array_equal(g, g[::-1])
    # a symmetric composition of a symmetric order-p method has order p+2
    # iff sum gamma^(p+1) = 0
    assert abs(np.sum(g ** (p + 1))) < 1e-14


@pytest.mark.parametrize("scheme,base", [(comp.TRIPLE_JUMP, 3), (comp.SUZUKI, 5)])
def test_substep_counts(scheme, base):
    for order in (2, 4, 6, 8):
        f = comp.schedule(order, scheme)
        assert len(f) == base ** (order // 2 - 1)
        assert abs(sum(f) - 1.0) < 1e-14
        assert f == f[::-1]


def _scalar(fractions, x):
    r = 1.0 + 0j
    for f in fractions:
        r *= (1 - 0.5j * f * x) / (1 + 0.5j * f * x)
    return r


@pytest.mark.parametrize("scheme", [comp.TRIPLE_JUMP, comp.SUZUKI])
@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_scalar_composed_cayley_has_the_order(scheme, order):
    f = comp.schedule(order, scheme)
    xs = np.geomspace(1e-4, 6.0, 160)
    err = np.array([abs(_scalar(f, x) - np.exp(-1j * x)) for x in xs])
    # asymptotic window: well above rounding, well below O(1)
    sel = (err > 1e-12) & (err < 1e-7)
    assert sel.sum() >= 5
    slope = np.polyfit(np.log(xs[sel]), np.log(err[sel]), 1)[0]
    assert abs(slope - (order + 1)) < 0.3
    for x in xs:
        assert abs(abs(_scalar(f, x)) - 1.0) < 2e-13


def test_trapezoidal_taylor_expansion_and_local_error():
    # Appendix A: U_trap(eps) = 1 - i eps H - (eps H)^2/2 + (i/4)(eps H)^3 + ...,
    # local error i (eps H)^3 / 12, here on H = [[1]] through the oracle's step
    g = GOLD["trapezoidal_taylor"]
    st = prop.DenseStepper(np.array([[1.0]]))
    eps = np.geomspace(1e-3, 2e-2, 12)
    u = np.array([st.trap(np.array([1.0 + 0j]), e)[0] for e in eps])
    A = np.vander(eps, 6, increasing=True)
    coef = np.linalg.lstsq(A, u, rcond=None)[0]
    want = [complex(a, b) for a, b in g["coefficients_of_epsH_powers"]]
    np.testing.assert_allclose(coef[:4], want, atol=1e-6)
    le = (u - np.exp(-1j * eps)) / eps ** 3
    assert abs(le[0] - complex(*g["local_error_cubic"])) < 1e-3


def test_implicit_euler_taylor_expansion():
    g = GOLD["implicit_euler_taylor"]
    st = prop.DenseStepper(np.array([[1.0]]))
    eps = np.geomspace(1e-3, 2e-2, 12)
    u = np.array([st.impl(np.array([1.0 + 0j]), e)[0] for e in eps])
    coef = np.linalg.lstsq(np.vander(eps, 6, increasing=True), u, rcond=None)[0]
    want = [complex(a, b) for a, b in g["coefficients_of_epsH_powers"]]
    np.testing.assert_allclose(coef[:4], want, atol=1e-4)


# ---------------------------------------------------------------------------
# "Optimal" compositions (Sec. II C) and the free-algebra order conditions


@pytest.mark.parametrize("scheme", [comp.TRIPLE_JUMP, comp.SUZUKI])
@pytest.mark.parametrize("order", [4, 6, 8])
def test_recursive_schemes_meet_the_general_order_conditions(scheme, order):
    g = comp.schedule(order, scheme)
    scale = sum(abs(x) for x in g) ** order
    assert comp.order_condition_residual(g, order) < 1e-14 * scale
    if order < 8:
        assert comp.order_condition_residual(g, order + 2) > 1e-6


@pytest.mark.parametrize("order,M,gmax", [(6, 9, 0.7985439909348300), (8, 17, 0.6055085338300345)])
def test_kahan_li_coefficients(order, M, gmax):
    g = comp.schedule(order, comp.OPTIMAL)
    assert len(g) == M
    assert abs(sum(g) - 1.0) < 1e-15
    assert g == g[::-1]
    assert abs(max(abs(x) for x in g) - gmax) < 1e-15
    # order exactly `order`: every condition up to that degree, not the next
    assert comp.order_condition_residual(g, order) < 1e-15
    assert comp.order_condition_residual(g, order + 2) > 1e-5
    # a wrong digit anywhere breaks the conditions
    for i in range(M // 2 + 1):
        bad = list(g)
        bad[i] += 1e-9
        bad[M - 1 - i] = bad[i]
        assert comp.order_condition_residual(bad, order) > 1e-10


def test_scalar_conditions_alone_do_not_pass_the_general_check():
    # a palindrome of M = 9 with sum 1, sum gamma^3 = sum gamma^5 = 0 meets the
    # scalar (commuting) conditions of order 6 but not the non-commutative one
    # at degree 5: the free-algebra check must see the difference
    from scipy.optimize import fsolve
    fixed = [0.3, 0.25]

    def eqs(v):
        g = comp.palindrome(fixed + list(v))
        return [sum(g) - 1.0, sum(x ** 3 for x in g), sum(x ** 5 for x in g)]

    v = fsolve(eqs, [-0.6, 0.1, 0.9], xtol=1e-13)
    g = comp.palindrome(fixed + list(v))
    assert max(abs(e) for e in eqs(v)) < 1e-13
    assert comp.order_condition_residual(g, 6) > 1e-4


@pytest.mark.parametrize("order", [6, 8])
def test_scalar_optimal_cayley_has_the_order(order):
    f = comp.schedule(order, comp.OPTIMAL)
    xs = np.geomspace(1e-3, 6.0, 160)
    err = np.array([abs(_scalar(f, x) - np.exp(-1j * x)) for x in xs])
    sel = (err > 1e-12) & (err < 1e-7)
    assert sel.sum() >= 5
    slope = np.polyfit(np.log(xs[sel]), np.log(err[sel]), 1)[0]
    assert abs(slope - (order + 1)) < 0.3
