"""Batched form: many independent avoided-crossing models of uneven grid
size and surface count in one persistent launch (captured as a CUDA graph),
and the S >= 3 diabatic -> adiabatic field builder, against the oracle."""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import FS, rel_l2
from oracle import fields as ofields, grid as ogrid, hamiltonian as oham, initial as oinit, propagate as oprop

pytestmark = pytest.mark.gpu


def _small_models(count, nmax=1024, base=1000):
    out, seed = [], base
    while len(out) < count:
        m = wl.avoided_crossing_model(seed)
        if m["N"] <= nmax:
            out.append(m)
        seed += 1
    return out


def _oracle_fields(m):
    if m["S"] == 2:
        return ofields.two_state(m["W"], m["dW"])
    V, F, _ = ofields.general_adiabatic(m["W"], m["dW"], m["S"])
    return V, F


def test_general_fields_vs_oracle(qglib, cuda):
    models = [m for m in _small_models(12, nmax=8192) if m["S"] == 3][:4]
    assert models
    for m in models:
        g = qglib.Grid([m["N"]], [m["qmin"]], [m["qmax"]])
        lm = qglib.Model(g, 3, [m["mass"]], W=m["W"], dW=m["dW"])
        Vg, Fg = lm.fields()
        V, F = _oracle_fields(m)
        assert np.abs(Vg - V).max() < 1e-13 * np.abs(V).max()
        assert np.abs(Fg - F).max() < 1e-9 * np.abs(F).max()


def test_batched_uneven_models_vs_oracle(qglib, cuda):
    models = _small_models(10, nmax=1024)
    assert {m["S"] for m in models} == {2, 3} and len({m["N"] for m in models}) > 1
    keep, states, wants = [], [], []
    dt, nsteps = 0.1 * FS, 2
    for m in models:
        g = qglib.Grid([m["N"]], [m["qmin"]], [m["qmax"]])
        lm = qglib.Model(g, m["S"], [m["mass"]], W=m["W"], dW=m["dW"])
        st = qglib.State(lm)
        st.set_gaussian(m["surface"], [m["q0"]], [m["p0"]], [m["sigma0"]])
        keep += [g, lm]
        states.append(st)
        V, F = _oracle_fields(m)
        q, dq = ogrid.points(m["qmin"], m["qmax"], m["N"])
        psi0 = oinit.state_on_surface(m["S"], m["surface"], oinit.gaussian([q], [m["q0"]], [m["p0"]], [m["sigma0"]]))
        H = oham.dense_h([m["qmin"]], [m["qmax"]], [m["N"]], [m["mass"]], V, F)
        wants.append(oprop.DenseStepper(H).propagate(psi0, dt, nsteps, oprop.MIDPOINT, 4, 1))
    batch = qglib.Batch(states)
    opts = qglib.default_solver_opts(tol=1e-14)
    batch.capture(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, dt, nsteps, opts)
    batch.replay()
    stt, stats = batch.stats()
    assert stt == [0] * len(models)
    for st, want, s in zip(states, wants, stats):
        assert rel_l2(st.get(), want) < 1e-11
        assert s["n_substeps"] == nsteps * 5


def test_graph_replay_equals_direct_run(qglib, cuda):
    models = _small_models(6, nmax=2048, base=2000)
    keep, a_states, b_states = [], [], []
    for m in models:
        g = qglib.Grid([m["N"]], [m["qmin"]], [m["qmax"]])
        lm = qglib.Model(g, m["S"], [m["mass"]], W=m["W"], dW=m["dW"])
        a, b = qglib.State(lm), qglib.State(lm)
        for s in (a, b):
            s.set_gaussian(m["surface"], [m["q0"]], [m["p0"]], [m["sigma0"]])
        keep += [g, lm]
        a_states.append(a)
        b_states.append(b)
    opts = qglib.default_solver_opts()
    A, B = qglib.Batch(a_states), qglib.Batch(b_states)
    A.capture(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, 0.1 * FS, 1, opts)
    for _ in range(3):
        A.replay()
    A.stats()
    B.run(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, 0.1 * FS, 3, opts)
    for a, b in zip(a_states, b_states):
        np.testing.assert_array_equal(a.get(), b.get())


def test_concurrent_propagate_calls_from_host_threads(qglib, cuda):
    # one qg_propagate per model from 8 host threads on 8 streams, grid sizes
    # mixed (each launch needs its own shared-memory size): every call
    # succeeds and equals the same call made alone
    import concurrent.futures as cf
    torch = cuda
    models = _small_models(16, nmax=8192, base=3000)
    keep, states, refs = [], [], []
    opts = qglib.default_solver_opts(tol=1e-13)
    for m in models:
        g = qglib.Grid([m["N"]], [m["qmin"]], [m["qmax"]])
        lm = qglib.Model(g, m["S"], [m["mass"]], W=m["W"], dW=m["dW"])
        a, b = qglib.State(lm), qglib.State(lm)
        for s in (a, b):
            s.set_gaussian(m["surface"], [m["q0"]], [m["p0"]], [m["sigma0"]])
        b.propagate(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, 0.1 * FS, 1, opts)
        keep += [g, lm]
        states.append(a)
        refs.append(b.get())
    streams = [torch.cuda.Stream() for _ in range(8)]
    for i, st in enumerate(states):
        st.set_stream(streams[i % 8])

    def lane(t):
        for st in states[t::8]:
            st.propagate(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, 0.1 * FS, 1, opts)

    with cf.ThreadPoolExecutor(8) as ex:
        list(ex.map(lane, range(8)))
    for st, ref in zip(states, refs):
        np.testing.assert_array_equal(st.get(), ref)
