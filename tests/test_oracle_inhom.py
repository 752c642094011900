"""Pins of the oracle's inhomogeneous coupling (`oracle.inhom`): free streaming and Strang
splitting around the homogeneous operator per cell.  CPU only.

* Free streaming of a drifting density wave f = (1 + eps cos(2 pi x / Lx)) M_T(v - u e1):
  the density is rho(x, t) = 1 + eps exp(-(2 pi t / Lx)^2 T / 2) cos(2 pi (x - u t) / Lx)
  (integrating the exact solution over v), which the cells' (2L)^3 Re fhat_0 must reproduce.
* Streaming by t and then -t is the identity; the total mass is kept.
* With a spatially uniform f the transport is the identity, so a Strang step is RK4 of the
  collision (Sec. 5.2) in every cell.
"""
import math

import numpy as np

import bz_inputs as bi
from oracle import inhom, kernels, spectral


def test_free_streaming_density_wave_closed_form():
    N, L, nx, Lx, eps, u, T = 32, 6.0, 8, 4.0, 0.3, 0.7, 0.5     # h = 2L/N small enough for the trapezoid rule
    f0 = bi.drifting_wave_samples(N, L, nx, Lx, eps, u, T)
    x = np.arange(nx) * Lx / nx
    for t in (0.0, 0.37, 1.1):
        rho = inhom.density(inhom.transport(f0, L, Lx, t), L)
        exact = 1 + eps * math.exp(-(2 * math.pi * t / Lx) ** 2 * T / 2) * np.cos(2 * math.pi * (x - u * t) / Lx)
        assert np.max(np.abs(rho - exact)) < 1e-12, (t, rho - exact)


def test_streaming_is_reversible_and_keeps_mass():
    N, L, nx, Lx = 8, 6.0, 8, 5.0
    f0 = bi.inhom_cells(N, L, nx, Lx)
    f1 = inhom.transport(f0, L, Lx, 0.8)
    assert abs(inhom.density(f1, L).sum() - inhom.density(f0, L).sum()) < 1e-12
    back = inhom.transport(f1, L, Lx, -0.8)
    assert np.max(np.abs(back - f0)) < 1e-12 * np.max(np.abs(f0))
    assert np.max(np.abs(f1 - f0)) > 1e-3 * np.max(np.abs(f0))          # it did move


def test_strang_on_uniform_f_is_rk4_per_cell():
    N, L, nx, Lx = 8, 6.0, 4, 5.0
    R = bi.R_from_L(L)
    plan = spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 2, 12)
    g = bi.random_mixture(N, L, seed=4, box=1.0)
    f0 = np.stack([g] * nx)
    got = inhom.strang(plan, f0, Lx, 0.1, 2)
    ref = spectral.rk4(plan, g, 0.1, 2)
    assert np.max(np.abs(got - ref[None])) < 1e-13 * np.max(np.abs(ref))


def test_strang_is_second_order():
    """Halving dt divides the splitting error by about four (Strang: streaming dt/2, collision
    dt, streaming dt/2), measured against a run with dt/8."""
    N, L, nx, Lx, T = 8, 6.0, 4, 3.0, 0.4
    R = bi.R_from_L(L)
    plan = spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 2, 12)
    f0 = bi.inhom_cells(N, L, nx, Lx, eps=0.3)
    ref = inhom.strang(plan, f0, Lx, T / 16, 16)
    e = [np.max(np.abs(inhom.strang(plan, f0, Lx, T / n, n) - ref)) for n in (2, 4)]
    print(f"Strang errors at dt = {T / 2}, {T / 4}: {e[0]:.2e}, {e[1]:.2e} (ratio {e[0] / e[1]:.2f})")
    assert 3.0 < e[0] / e[1] < 5.5
