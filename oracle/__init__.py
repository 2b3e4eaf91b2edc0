"""Plain, slow FP64 CPU oracle for the composed implicit propagation method.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check in
__graft_entry__ and the CPU-baseline leg of bench.py may import anything from
this package.  The CUDA library never calls it and shares no code with it.

Everything here is the plain definition of what the method computes, written
in the paper's notation with dense matrices:

* grid.py         -- Fourier grid, explicit DFT matrix, spectral derivative
                     (dynamic Fourier method, Sec. II D)
* hamiltonian.py  -- dense adiabatic Hamiltonian, Eq. (adiab_mol_ham)
* fields.py       -- diabatic -> adiabatic potential and coupling for two
                     states (Eqs. pot_diab2adiab, ..._orthogonal_transformation,
                     nonadiab_c), evaluated in 50-digit arithmetic
* initial.py      -- Gaussian initial state (Sec. III)
* composition.py  -- triple-jump / Suzuki coefficients and the recursive
                     composition (Eqs. triple_jump, suzukis_fractal, Sec. II C)
* propagate.py    -- explicit/implicit Euler, trapezoidal rule and implicit
                     midpoint (Eqs. exp_euler, imp_euler, trap_rule,
                     imp_midpoint) with dense LU solves, compositions
* observables.py  -- inner product, norm, populations, energy, symplectic form
                     (Sec. II A)
* representation.py -- diabatic Hamiltonian, psi = O^T psi_diab (Sec. II E),
                     trigonometric interpolation between grids (Appendix B)
* cpu_baseline/   -- the same algorithm as the GPU library in plain C with
                     OpenMP (a timing baseline, pinned to the dense oracle)

Conventions (the paper leaves them open; each is a stated reading):
hbar = 1; grid q_j = qmin + j*dq, dq = (qmax - qmin)/N, periodic;
k_j = 2 pi/(N dq) * (j if j < N/2 else j - N); inner product
<a|b> = dq * sum_s sum_j conj(a_s(q_j)) b_s(q_j) (product of dq over dimensions);
adiabatic surfaces in ascending energy (index 0 = ground);
state layout (S, N_1, ..., N_D), C order.
"""
from . import composition, grid, hamiltonian, fields, initial, propagate, observables, representation  # noqa: F401
