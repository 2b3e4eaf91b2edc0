"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package holds no arithmetic of the propagation method: it only produces
input data (grids' extents, diabatic model curves and their derivatives,
initial-state parameters, random test vectors).  Everything the method
computes from these inputs -- adiabatic fields, initial Gaussians, the
Hamiltonian action, Krylov solves, compositions, observables -- is implemented
separately by the oracle and by the CUDA library.

Units: Hartree atomic units (hbar = 1, electron mass = 1), as in Sec. III.
"""
from .constants import (AU_TIME_PER_FS, NAI_REDUCED_MASS, NAI_QMIN, NAI_QMAX,
                        NAI_N, NAI_Q0, NAI_P0, NAI_SIGMA0, NAI_TF,
                        PHI_Q0, PHI_P0)
from .nai_like import nai_like_diabatic, nai_like_params, initial_gaussian_params
from .random_inputs import random_psi, random_adiabatic_fields
from .avoided_crossing import avoided_crossing_model
from .model2d import PARAMS as MODEL2D_PARAMS, model2d_diabatic, model2d_initial
