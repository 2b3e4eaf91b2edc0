"""2-D grids under every work split of the cooperative launch: the shared-
memory FFT batch chunked over several passes (few CTAs, many rows each) and
the FFT tables kept in global memory (grids too long for the shared-memory
copy) must give the same H psi and the same steps as the default split."""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import FS, rel_l2
from oracle import grid as ogrid

pytestmark = pytest.mark.gpu


def _random_model(qg, ns, S=2, seed=71):
    qmin, qmax, mass = [-3.0, -2.0], [3.0, 2.5], [2000.0, 3000.0]
    V, F = wl.random_adiabatic_fields(S, 2, ns, seed=seed, v_scale=0.05, f_scale=0.3)
    g = qg.Grid(list(ns), qmin, qmax)
    return g, qg.Model(g, S, mass, V=V, F=F), (qmin, qmax, mass)


@pytest.mark.parametrize("ns,widths", [((512, 256), (0, 8, 3)), ((256, 512), (0, 16, 5))])
def test_hpsi_and_steps_independent_of_launch_width(qglib, cuda, ns, widths):
    g, m, _ = _random_model(qglib, ns)
    psi = wl.random_psi(2, ns, seed=72, smooth=12)
    psi /= np.sqrt(np.sum(np.abs(psi) ** 2) * np.prod([(g.qmax[d] - g.qmin[d]) / ns[d] for d in range(2)]))
    hs, outs = [], []
    for w in widths:
        st = qglib.State(m)
        st.set_launch_width(w)
        st.set(psi)
        hs.append(st.apply_h())
        st.propagate(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, 0.02 * FS, 2, qglib.default_solver_opts(tol=1e-14, solver=1))
        outs.append(st.get())
    for k in range(1, len(widths)):
        assert rel_l2(hs[k], hs[0]) < 1e-13, (widths[k], rel_l2(hs[k], hs[0]))
        assert rel_l2(outs[k], outs[0]) < 1e-12, (widths[k], rel_l2(outs[k], outs[0]))


def test_long_grid_tables_in_global_memory(qglib, cuda):
    # 4096 x 256: the FFT tables (36 bytes per point of n0 + n1) no longer fit
    # beside the other shared arrays, so the transforms read them from global
    # memory.  Plane waves are eigenvectors of the kinetic operator.
    ns = (4096, 256)
    g = qglib.Grid(list(ns), [0.0, 0.0], [40.0, 3.0])
    m = qglib.Model(g, 2, [3.0, 5.0], V=np.zeros((2,) + ns), F=np.zeros((2, 1) + ns))
    st = qglib.State(m)
    q1 = ogrid.points(0.0, 40.0, ns[0])[0]
    q2 = ogrid.points(0.0, 3.0, ns[1])[0]
    k1 = ogrid.wavenumbers(0.0, 40.0, ns[0])[1001]
    k2 = ogrid.wavenumbers(0.0, 3.0, ns[1])[-17]
    pw = np.exp(1j * (k1 * q1[:, None] + k2 * q2[None, :]))
    st.set(np.stack([0 * pw, pw]))
    got = st.apply_h()
    want = (k1 ** 2 / 6.0 + k2 ** 2 / 10.0) * pw
    assert np.abs(got[1] - want).max() < 1e-10 * np.abs(want).max()
    assert np.abs(got[0]).max() < 1e-10 * np.abs(want).max()


def test_stiff_lanczos_matches_gmres_and_conserves_norm(qglib, cuda):
    # random fields, light masses: about 45 Krylov iterations per solve.  A
    # short-recurrence solver whose normalisation drifts loses unitarity here
    # long before it fails to "converge" on its own residual estimate.
    ns = (512, 256)
    g, m, (qmin, qmax, _) = _random_model(qglib, ns)
    psi = wl.random_psi(2, ns, seed=72, smooth=12)
    dv = np.prod([(qmax[d] - qmin[d]) / ns[d] for d in range(2)])
    psi /= np.sqrt(np.sum(np.abs(psi) ** 2) * dv)
    out = {}
    for solver in (0, 1):
        st = qglib.State(m)
        st.set(psi)
        s = st.propagate(qglib.QG_MIDPOINT, 4, qglib.QG_SUZUKI, 0.02 * FS, 2,
                         qglib.default_solver_opts(tol=1e-14, solver=solver))
        out[solver] = st.get()
        print("solver %d: krylov/substep %.1f, norm - 1 = %.2e" % (solver, s["n_krylov"] / s["n_substeps"],
                                                                  st.norm() - 1.0))
        assert abs(st.norm() - 1.0) < 1e-12
    assert rel_l2(out[1], out[0]) < 1e-11
