"""GB300 (sm_103a) library for composed implicit propagation of multi-surface
nuclear wavepackets in the adiabatic representation (arXiv:1902.04661).

The compute path is libqgeom.so (hand-written CUDA, C-ABI in include/qgeom.h);
this package is its ctypes binding.  Build it with build.build()."""
from ._binding import *  # noqa: F401,F403
from ._binding import (Grid, Model, State, SolverOpts, StepStats, QgError, QgLibraryMissing,  # noqa: F401
                       default_solver_opts, qg_batch_propagate, Batch, qg_version, lib, LIB_PATH, EXPORTED)
