"""Pins of the oracle's real-data reading (`real_band`, `collide_real`): f is a real function
(Sec. 2), so its coefficients are Hermitian, fhat_{-k} = conj fhat_k, except on the Nyquist
planes (signed index -N/2, no partner +N/2), which the reading drops.  CPU only.

* `real_band` is the identity on the coefficients of a real grid function whose Nyquist
  planes are zero (numpy's FFT makes them), gives real grid values for any input, and
  removes a purely imaginary f.
* `collide_real` equals the O(N^6) double sum of eq. sum (eq. approxG weights) applied to
  the band (N = 8), and equals the circular operator on a real f without Nyquist content.
* Off the Nyquist planes its result is Hermitian for any input (F(-k) = conj F(k)); on them
  the weight alpha_p(k) at the signed index -N/2 has no mirror, so Q need not be.
* For a smooth real f (BKW, Sec. 5.1) it differs from the circular operator by less than the
  Nyquist content of f allows.
"""
import numpy as np
import pytest

import bz_inputs as bi
from oracle import kernels, spectral


def _real_grid_band(N, seed):
    u = bi.SplitMix64(seed).uniform(N ** 3).reshape(N, N, N)
    fh = np.fft.fftn(u - 0.5) / N ** 3
    fh[spectral.nyquist_mask(N)] = 0
    return fh


def test_real_band_identity_realness_and_imaginary_part():
    for N in (8, 12):
        fh = _real_grid_band(N, seed=N)
        assert np.max(np.abs(spectral.real_band(fh) - fh)) < 1e-15
        x = bi.random_fhat(N, seed=100 + N)
        g = np.fft.ifftn(spectral.real_band(x))
        assert np.max(np.abs(g.imag)) < 1e-15 * max(1.0, np.max(np.abs(g.real))) + 1e-17
        assert np.max(np.abs(spectral.real_band(1j * fh))) < 1e-15
        assert np.all(spectral.real_band(x)[spectral.nyquist_mask(N)] == 0)
        assert np.sum(spectral.nyquist_mask(N)) == N ** 3 - (N - 1) ** 3


@pytest.fixture(scope="module")
def plan8():
    L = 6.0
    return spectral.OraclePlan(8, L, bi.R_from_L(L), -1.0, kernels.Kernel("family", 0.5), 3, 12)


def test_collide_real_equals_direct_sum_of_the_band(plan8):
    f = bi.random_fhat(8, seed=5)
    Q = spectral.collide_real(plan8, f)
    D = spectral.direct_sum(plan8, spectral.real_band(f))
    assert np.max(np.abs(Q - D)) < 1e-12 * np.max(np.abs(D))
    fr = _real_grid_band(8, seed=6)                    # real f, no Nyquist content
    Qc = spectral.collide(plan8, fr)
    assert np.max(np.abs(spectral.collide_real(plan8, fr) - Qc)) < 1e-14 * np.max(np.abs(Qc))


def test_collide_real_is_hermitian_off_the_nyquist_planes(plan8):
    ny = spectral.nyquist_mask(8)
    for seed in (1, 2):
        Q = spectral.collide_real(plan8, bi.random_fhat(8, seed=seed))
        d = np.abs(spectral.mirror(Q) - np.conj(Q))
        assert np.max(d[~ny]) < 1e-13 * np.max(np.abs(Q))
        assert np.max(d[ny]) > 1e-6 * np.max(np.abs(Q))      # alpha at -N/2 has no mirror


def test_term_ranges_add_up(plan8):
    f = bi.random_fhat(8, seed=9)
    full = spectral.collide_real(plan8, f)
    parts = spectral.collide_real(plan8, f, 0, 10) + spectral.collide_real(plan8, f, 10, plan8.P)
    assert np.max(np.abs(parts - full)) < 1e-13 * np.max(np.abs(full))


def test_smooth_real_f_is_barely_changed():
    """BKW at t = 6.5 on N = 32 (L = 6.62): its Nyquist planes hold |fhat| ~ 5e-8 of fhat_0, and
    the real-data reading moves Q by a few 1e-7 of max|Q| (at N = 16 the same f is
    under-resolved: Nyquist content 1e-2, and Q moves by 5%)."""
    N, R = 32, 6.0
    L = bi.L_from_R(R)
    f = bi.bkw_fhat(N, L, bi.bkw_K(6.5))
    ny = spectral.nyquist_mask(N)
    content = np.max(np.abs(f[ny])) / abs(f[0, 0, 0])
    assert np.max(np.abs(spectral.real_band(f) - np.where(ny, 0, f))) < 1e-15 * abs(f[0, 0, 0])   # f is real
    plan = spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 4, 12)
    Q = spectral.collide(plan, f, 0, 8)
    Qr = spectral.collide_real(plan, f, 0, 8)
    dev = np.max(np.abs(Q - Qr)) / np.max(np.abs(Q))
    print(f"Nyquist content {content:.2e}, |Q - Q_real| / max|Q| = {dev:.2e}")
    assert content < 1e-7 and dev < 1e-5
