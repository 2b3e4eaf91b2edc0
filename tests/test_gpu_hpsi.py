"""GPU parity of the fused H psi pass (Eq. adiab_mol_ham, dynamic Fourier
method of Sec. II D) and of the model / initial-state builders, against the
CPU oracle on identical seeded inputs."""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import nai_inputs, nai_library_model, nai_oracle_fields, rel_l2
from oracle import fields as ofields, grid as ogrid, hamiltonian as oham, initial as oinit

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,S", [(8, 2), (16, 3), (32, 4), (64, 2), (128, 2), (256, 3), (512, 2), (1024, 2), (1024, 4)])
def test_hpsi_random_fields_vs_dense_oracle(qglib, cuda, n, S):
    qmin, qmax, mass = -2.0, 9.0, 13.0
    V, F = wl.random_adiabatic_fields(S, 1, (n,), seed=100 + n + S)
    psi = wl.random_psi(S, (n,), seed=200 + n + S)
    g = qglib.Grid([n], [qmin], [qmax])
    m = qglib.Model(g, S, [mass], V=V, F=F)
    st = qglib.State(m)
    st.set(psi)
    got = st.apply_h()
    H = oham.dense_h([qmin], [qmax], [n], [mass], V, F)
    want = oham.apply_h(H, psi)
    assert rel_l2(got, want) < 1e-12


@pytest.mark.parametrize("n", [2048, 4096, 8192])
def test_hpsi_nai_like_full_size_vs_matrix_free_oracle(qglib, cuda, n):
    grid, model = nai_library_model(qglib, n)
    V, F = nai_oracle_fields(n)
    psi = wl.random_psi(2, (n,), seed=7 + n, smooth=n // 8)
    st = qglib.State(model)
    st.set(psi)
    got = st.apply_h()
    want = oham.apply_h_matrix_free(wl.NAI_QMIN, wl.NAI_QMAX, n, wl.NAI_REDUCED_MASS, V, F, psi)
    assert rel_l2(got, want) < 1e-12


@pytest.mark.parametrize("n", [8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192])
def test_hpsi_plane_waves_free_particle(qglib, cuda, n):
    """Every transform plan (radix-8 and radix-4 passes, the factored FP64
    passes from N = 16 on): on a grid plane wave e^{ikq} with V = F = 0, H psi
    = k^2 / 2m psi exactly, the Nyquist wave included.  The bound is the
    rounding of a length-n transform, log2(n) eps times the largest k^2 / 2m."""
    qmin, mass = 0.0, 3.0
    qmax = 0.05 * n
    g = qglib.Grid([n], [qmin], [qmax])
    m = qglib.Model(g, 2, [mass], V=np.zeros((2, n)), F=np.zeros((1, 1, n)))
    st = qglib.State(m)
    k = ogrid.wavenumbers(qmin, qmax, n)
    emax = np.max(k ** 2) / (2 * mass)
    tol = 1e-13 + 2e-14 * np.log2(n) * emax
    p = np.arange(n)

    def wave(j):
        # e^{i k_j q_p} = e^{2 pi i j p / n} (qmin = 0), the phase reduced
        # exactly in integers: exp of k q itself would carry the rounding of
        # k q (up to ~3000 rad here), which the k^2 multiplier amplifies
        return np.exp(2j * np.pi * ((j * p) % n) / n)

    for j in sorted({0, 1, 5 % n, n // 2 - 1, n // 2, n - 1}):
        psi = np.stack([wave(j), wave((j + 3) % n)])
        st.set(psi)
        got = st.apply_h()
        want = np.stack([k[j] ** 2 / (2 * mass) * psi[0], k[(j + 3) % n] ** 2 / (2 * mass) * psi[1]])
        assert np.abs(got - want).max() < tol, (n, j, np.abs(got - want).max(), tol)


def test_model_fields_from_diabatic_vs_oracle(qglib, cuda):
    n = 2048
    grid, model = nai_library_model(qglib, n)
    Vg, Fg = model.fields()
    V, F = nai_oracle_fields(n)
    assert np.abs(Vg - V).max() < 1e-15 + 1e-14 * np.abs(V).max()
    assert np.abs(Fg - F).max() < 1e-12 * np.abs(F).max()


def test_gaussian_initial_state_vs_oracle(qglib, cuda):
    n = 2048
    grid, model = nai_library_model(qglib, n)
    st = qglib.State(model)
    for seed in (None, 0, 3):
        q0, p0, s0 = wl.initial_gaussian_params(seed)
        st.set_gaussian(1, [q0], [p0 + 1.5], [s0])
        q, dq = ogrid.points(wl.NAI_QMIN, wl.NAI_QMAX, n)
        want = oinit.state_on_surface(2, 1, oinit.gaussian([q], [q0], [p0 + 1.5], [s0]))
        assert rel_l2(st.get(), want) < 1e-13


def test_observables_vs_oracle(qglib, cuda):
    from oracle import observables as oobs
    n = 512
    qmin, qmax, mass = -5.0, 5.0, 50.0
    V, F = wl.random_adiabatic_fields(3, 1, (n,), seed=5)
    psi = wl.random_psi(3, (n,), seed=6, smooth=40)
    phi = wl.random_psi(3, (n,), seed=8, smooth=40)
    g = qglib.Grid([n], [qmin], [qmax])
    m = qglib.Model(g, 3, [mass], V=V, F=F)
    a, b = qglib.State(m), qglib.State(m)
    a.set(psi)
    b.set(phi)
    dq = (qmax - qmin) / n
    H = oham.dense_h([qmin], [qmax], [n], [mass], V, F)
    assert abs(a.norm() - oobs.norm(psi, dq)) < 1e-13 * oobs.norm(psi, dq)
    np.testing.assert_allclose(a.population(), oobs.populations(psi, dq), rtol=1e-13)
    e = oobs.energy(H, psi, dq)
    assert abs(a.energy() - e) < 1e-12 * abs(e)
    ov = oobs.inner(psi, phi, dq)
    assert abs(a.overlap(b) - ov) < 1e-13 * abs(ov)
