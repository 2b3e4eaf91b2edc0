"""Seeded random test inputs (input data only)."""
import numpy as np


def random_psi(S, grid_shape, seed, smooth=None):
    """Complex128 array of shape (S, *grid_shape) with N(0,1) real and imaginary
    parts (PCG64).  If smooth is an integer, only Fourier modes |m| <= smooth
    along every axis are kept, giving a band-limited smooth field."""
    rng = np.random.default_rng(seed)
    shape = (S,) + tuple(grid_shape)
    psi = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if smooth is not None:
        spec = np.fft.fftn(psi, axes=tuple(range(1, len(shape))))
        for ax, n in enumerate(grid_shape, start=1):
            m = np.fft.fftfreq(n, 1.0 / n)
            keep = (np.abs(m) <= smooth).astype(float)
            sh = [1] * len(shape)
            sh[ax] = n
            spec = spec * keep.reshape(sh)
        psi = np.fft.ifftn(spec, axes=tuple(range(1, len(shape))))
    return np.ascontiguousarray(psi)


def random_adiabatic_fields(S, D, grid_shape, seed, v_scale=0.1, f_scale=0.5):
    """Seeded random adiabatic potential V (S, *grid) and couplings F
    (D, S(S-1)/2, *grid) (upper triangle, F_ji = -F_ij implied)."""
    rng = np.random.default_rng(seed)
    V = v_scale * rng.standard_normal((S,) + tuple(grid_shape))
    npair = S * (S - 1) // 2
    F = f_scale * rng.standard_normal((D, npair) + tuple(grid_shape))
    return np.ascontiguousarray(V), np.ascontiguousarray(F)
