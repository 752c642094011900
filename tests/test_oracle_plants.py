"""Planted mistakes in the oracle must make at least one pin fail (CPU only).

Each test plants one plausible mistake into the oracle (monkeypatched) and checks
that the pin guarding that part no longer passes.
"""
import math

import numpy as np

import bz_inputs as bi
from oracle import ftable, kernels, spectral


def _bkw_err(plan, N, L):
    K = bi.bkw_K(6.5)
    Q = spectral.collide(plan, bi.bkw_fhat(N, L, K))
    return np.max(np.abs(spectral.to_grid(Q, L) - spectral.bkw_Q(spectral.grid_v2(N, L), K)))


def _plan(N=16, kern=None):
    R = 6.0
    L = bi.L_from_R(R)
    return spectral.OraclePlan(N, L, R, 0.0, kern or kernels.Kernel("family", 0.5), 16, 12), L


def test_pin_baseline_passes():
    plan, L = _plan()
    assert _bkw_err(plan, 16, L) < 3e-3


def test_plant_wrong_twiddle_sign_breaks_bkw_pin(monkeypatch):
    plan, L = _plan()
    orig = spectral.OraclePlan.beta
    monkeypatch.setattr(spectral.OraclePlan, "beta", lambda self, p: np.conj(orig(self, p)))
    assert _bkw_err(plan, 16, L) > 3e-3


def test_plant_missing_normalisation_breaks_bkw_pin(monkeypatch):
    plan, L = _plan()
    orig = spectral.OraclePlan.alpha
    monkeypatch.setattr(spectral.OraclePlan, "alpha", lambda self, p: orig(self, p) * 16 ** 3)
    assert _bkw_err(plan, 16, L) > 3e-3


def test_plant_radial_power_breaks_bkw_pin():
    plan, L = _plan()
    plan.c = plan.wr * plan.wq * plan.r          # |q|^(d-2) instead of |q|^(d-1)
    assert _bkw_err(plan, 16, L) > 3e-3


def test_plant_dropped_taylor_term_breaks_series_pin(monkeypatch):
    kern = kernels.Kernel("family", 0.5)
    orig = kernels.Kernel.taylor_moments
    monkeypatch.setattr(kernels.Kernel, "taylor_moments",
                        lambda self, eps: orig(self, eps)[:2] + (0.0,))
    L, N, r, q = 10.0, 16, 7.0, np.array([0.0, 0.6, 0.8])
    kv = np.array([7, 7, -8])
    got = ftable.fentries(N, L, kv[None], np.array([r]), q[None], kern)[0]
    ex = ftable.f_exact_series(kv, r, q, L, kern)
    z = math.pi * r / (2 * L) * np.linalg.norm(kv)
    assert abs(got - ex) > ftable.taylor_remainder_bound(z, kern)


def test_plant_transposed_axis_breaks_library_dft_pin(monkeypatch):
    x = bi.random_fhat(6, seed=3)

    def bad(x, sign):
        W = spectral.dft_matrix(x.shape[0], sign)
        y = np.einsum("ab,bcd->acd", W, x)
        y = np.einsum("cb,abd->acd", W, y)
        return np.einsum("db,acb->adc", W, y)   # last two axes swapped
    assert not np.allclose(bad(x, -1), np.fft.fftn(x), atol=1e-9)


def test_plant_real_band_without_conjugate_breaks_identity_pin(monkeypatch):
    """real_band with the mirror taken without conjugation is not the identity on a real f."""
    N = 8
    u = bi.SplitMix64(3).uniform(N ** 3).reshape(N, N, N)
    fh = np.fft.fftn(u - 0.5) / N ** 3
    fh[spectral.nyquist_mask(N)] = 0
    assert np.max(np.abs(spectral.real_band(fh) - fh)) < 1e-15

    def bad(f):
        f = np.asarray(f, dtype=np.complex128)
        out = 0.5 * (f + spectral.mirror(f))
        out[spectral.nyquist_mask(f.shape[0])] = 0.0
        return out
    monkeypatch.setattr(spectral, "real_band", bad)
    assert np.max(np.abs(spectral.real_band(fh) - fh)) > 1e-6


def test_plant_streaming_phase_sign_breaks_density_wave_pin(monkeypatch):
    """Free streaming with the phase conjugated moves the drifting wave the wrong way."""
    from oracle import inhom
    N, L, nx, Lx, eps, u, T, t = 32, 6.0, 8, 4.0, 0.3, 0.7, 0.5, 0.37
    f0 = bi.drifting_wave_samples(N, L, nx, Lx, eps, u, T)
    x = np.arange(nx) * Lx / nx
    exact = 1 + eps * math.exp(-(2 * math.pi * t / Lx) ** 2 * T / 2) * np.cos(2 * math.pi * (x - u * t) / Lx)
    assert np.max(np.abs(inhom.density(inhom.transport(f0, L, Lx, t), L) - exact)) < 1e-12
    monkeypatch.setattr(inhom, "transport", _transport_flipped)
    assert np.max(np.abs(inhom.density(inhom.transport(f0, L, Lx, t), L) - exact)) > 1e-3


def _transport_flipped(fcells, L, Lx, t):
    from oracle import inhom
    nx, N = fcells.shape[0], fcells.shape[1]
    fv = np.stack([spectral.to_grid(fcells[c], L) for c in range(nx)])
    v1 = -L + 2.0 * L * np.arange(N) / N
    kappa = spectral.signed(nx).astype(np.float64)
    gx = np.einsum("ab,bijk->aijk", inhom._x_dft_matrix(nx, -1), fv)
    gx = gx * np.exp(+2j * math.pi * np.outer(kappa, v1) * t / Lx)[:, :, None, None]     # wrong sign
    fv = np.einsum("ab,bijk->aijk", inhom._x_dft_matrix(nx, +1), gx) / nx
    return np.stack([inhom._to_coeffs(fv[c]) for c in range(nx)])
