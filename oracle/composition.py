"""Composition coefficients and recursive symmetric composition (Sec. II C).

Eq. (triple_jump): M = 3, gamma_1 = gamma_3 = 1/(2 - 2^{1/(p+1)}),
                   gamma_2 = -2^{1/(p+1)}/(2 - 2^{1/(p+1)}).
Eq. (suzukis_fractal): M = 5, gamma_1 = gamma_2 = gamma_4 = gamma_5
                   = 1/(4 - 4^{1/(p+1)}), gamma_3 = -4^{1/(p+1)}/(4 - 4^{1/(p+1)}).
Recursion (Sec. II C): U_{p+2}(dt) = U_p(gamma_M dt) ... U_p(gamma_1 dt),
with the gammas of the inner order p; order 2 is the elementary method.
"""
TRIPLE_JUMP = 0
SUZUKI = 1
OPTIMAL = 2

# Non-recursive "optimal" symmetric compositions (Sec. II C): Kahan and Li
# (1997) minimise max|gamma_n| at the smallest M beyond the minimum -- M = 9
# for order 6, M = 17 for order 8.  The coefficients are not printed in the
# paper; these are Kahan and Li's published values (first half of each
# palindrome, middle coefficient last).  Order 4 uses Suzuki's fractal, which
# Sec. II C names the optimal fourth-order scheme.
KAHAN_LI_HALF = {
    6: [0.39216144400731413927925056, 0.33259913678935943859974864,
        -0.70624617255763935980996482, 0.08221359629355080023149045,
        0.79854399093482996339895035],
    8: [0.13020248308889008087881763, 0.56116298177510838456196441,
        -0.38947496264484728640807860, 0.15884190655515560089621075,
        -0.39590389413323757733623154, 0.18453964097831570709183254,
        0.25837438768632204729397911, 0.29501172360931029887096624,
        -0.60550853383003451169892108],
}


def palindrome(half):
    """gamma_1..gamma_M from the first half and the middle coefficient."""
    return list(half) + list(half[-2::-1])


def gammas(scheme, p):
    """Coefficients gamma_1..gamma_M that raise a symmetric order-p method to p+2."""
    if scheme == TRIPLE_JUMP:
        r = 2.0 ** (1.0 / (p + 1))
        g1 = 1.0 / (2.0 - r)
        g2 = -r / (2.0 - r)
        return [g1, g2, g1]
    if scheme == SUZUKI:
        r = 4.0 ** (1.0 / (p + 1))
        g1 = 1.0 / (4.0 - r)
        g3 = -r / (4.0 - r)
        return [g1, g1, g3, g1, g1]
    raise ValueError("unknown composition scheme %r" % (scheme,))


def schedule(order, scheme):
    """Flat list of sub-step fractions of dt, in the order they are applied.

    U_{p+2}(dt) applies U_p(gamma_1 dt) first and U_p(gamma_M dt) last; each
    U_p(gamma_n dt) expands into the order-p list scaled by gamma_n.  The
    OPTIMAL scheme is one non-recursive list (orders 6, 8; order 4 and 2 as
    SUZUKI)."""
    if order < 2 or order % 2:
        raise ValueError("order must be an even integer >= 2")
    if scheme == OPTIMAL:
        if order in KAHAN_LI_HALF:
            return palindrome(KAHAN_LI_HALF[order])
        if order > 8:
            raise ValueError("no optimal composition of order %d" % order)
        scheme = SUZUKI
    flat = [1.0]
    p = 2
    while p < order:
        flat = [g * f for g in gammas(scheme, p) for f in flat]
        p += 2
    return flat


# ---------------------------------------------------------------------------
# Order conditions of a symmetric composition of a symmetric second-order
# method, checked in the free algebra.  A symmetric method has the modified
# generator log Phi(h) = h Y1 + h^3 Y3 + h^5 Y5 + ... with free,
# non-commuting Y_k (only odd powers: symmetry).  The composition
# Psi(h) = Phi(gamma_M h) ... Phi(gamma_1 h) has order p iff Psi(h) and
# exp(h Y1) agree in every word of the Y's of degree <= p (degree of Y_k is
# k).  Elements are dicts word -> coefficient, words tuples of degrees,
# products truncated above degree p.


def _words_mul(a, b, p):
    out = {}
    for wa, ca in a.items():
        da = sum(wa)
        for wb, cb in b.items():
            if da + sum(wb) > p:
                continue
            w = wa + wb
            out[w] = out.get(w, 0.0) + ca * cb
    return out


def _words_exp(x, p):
    """exp(x) truncated at degree p, for x without a constant term."""
    out = {(): 1.0}
    term = {(): 1.0}
    for n in range(1, p + 1):
        term = _words_mul(term, x, p)
        term = {w: c / n for w, c in term.items()}
        if not term:
            break
        for w, c in term.items():
            out[w] = out.get(w, 0.0) + c
    return out


def order_condition_residual(gammas_list, p):
    """Largest |coefficient| of Psi - exp(Y1) over the words of degree <= p
    (0 up to rounding iff the composition has order >= p)."""
    odd = [k for k in range(1, p + 1, 2)]
    psi = {(): 1.0}
    for g in gammas_list:
        phi = _words_exp({(k,): g ** k for k in odd}, p)
        psi = _words_mul(phi, psi, p)
    ref = _words_exp({(1,): 1.0}, p)
    keys = set(psi) | set(ref)
    return max(abs(psi.get(w, 0.0) - ref.get(w, 0.0)) for w in keys)
