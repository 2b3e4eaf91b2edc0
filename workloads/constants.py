"""Numbers that define the synthetic NaI-like workloads.

Printed in Sec. III (NaI example): the grid of 2048 points on [3.8, 47.0) a.u.,
the initial Gaussian (q0 = 4.9889 a.u., p0 = 0, sigma0 = 0.110436 a.u.), the
final time t_f = 10500 a.u., and the second Gaussian used for the symplectic
form (q0 = 5.05 a.u., p0 = 2.5 a.u., same sigma0; Fig. 6 caption).
The paper does not print the reduced mass; it is computed here from standard
atomic masses of 23Na and 127I (CODATA/AME values) and the atomic mass unit
in electron masses.
"""
AU_TIME_PER_FS = 41.341373335182          # 1 fs in atomic units of time
AMU_IN_ME = 1822.888486209                # 1 u in electron masses
_M_NA_U = 22.98976928
_M_I_U = 126.904473
NAI_REDUCED_MASS = _M_NA_U * _M_I_U / (_M_NA_U + _M_I_U) * AMU_IN_ME

NAI_QMIN = 3.8
NAI_QMAX = 47.0
NAI_N = 2048
NAI_Q0 = 4.9889
NAI_P0 = 0.0
NAI_SIGMA0 = 0.110436
NAI_TF = 10500.0
PHI_Q0 = 5.05
PHI_P0 = 2.5
