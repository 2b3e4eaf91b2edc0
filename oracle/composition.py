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
    U_p(gamma_n dt) expands into the order-p list scaled by gamma_n."""
    if order < 2 or order % 2:
        raise ValueError("order must be an even integer >= 2")
    flat = [1.0]
    p = 2
    while p < order:
        flat = [g * f for g in gammas(scheme, p) for f in flat]
        p += 2
    return flat
