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
