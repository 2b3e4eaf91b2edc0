"""Shared set-up for the GPU parity tests: models on the library side and the
same inputs on the oracle side (inputs come only from workloads/)."""
import numpy as np

import workloads as wl
from oracle import fields as ofields, grid as ogrid

FS = wl.AU_TIME_PER_FS


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def nai_inputs(n, qmin=wl.NAI_QMIN, qmax=wl.NAI_QMAX):
    q, dq = ogrid.points(qmin, qmax, n)
    W, dW = wl.nai_like_diabatic(q)
    return q, dq, W, dW


def nai_library_model(qg, n, qmin=wl.NAI_QMIN, qmax=wl.NAI_QMAX):
    q, dq, W, dW = nai_inputs(n, qmin, qmax)
    grid = qg.Grid([n], [qmin], [qmax])
    model = qg.Model(grid, 2, [wl.NAI_REDUCED_MASS], W=W, dW=dW)
    return grid, model


def nai_oracle_fields(n, qmin=wl.NAI_QMIN, qmax=wl.NAI_QMAX):
    q, dq, W, dW = nai_inputs(n, qmin, qmax)
    return ofields.two_state(W, dW)
