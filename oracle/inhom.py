"""The spatially inhomogeneous equation df/dt + v_1 df/dx = Q(f, f) on a periodic interval
[0, Lx) of n_x cells (x_c = c Lx / n_x) with the homogeneous solver as a black box per cell
(the closing remark of the paper, Sec. 6: the method can serve the nonhomogeneous equation).
The paper gives no scheme for this; the reading here is Strang splitting.  Oracle: test
infrastructure, FP64, shares no code with the CUDA library.

* `transport(fcells, L, Lx, t)`: exact free streaming f(x, v, t) = f(x - v_1 t, v) at the
  velocity nodes v_j = -L + 2 L j / N, spectral in x: the grid values of every cell
  (`spectral.to_grid`), an x-DFT at every velocity node, the phase exp(-2 pi i kappa v_1 t / Lx)
  with the signed x-mode kappa in {-n_x/2, ..., n_x/2 - 1}, the inverse x-DFT, and the
  coefficients again (the 3D DFT of the grid values, divided by N^3).
* `strang(plan, fcells, Lx, dt, nsteps)`: per step, transport dt/2, RK4 (Sec. 5.2) of the
  collision over dt in every cell (`spectral.rk4`), transport dt/2.
"""
from __future__ import annotations

import math

import numpy as np

from . import spectral


def _x_dft_matrix(nx: int, sign: int) -> np.ndarray:
    a = np.arange(nx)
    return np.exp(sign * 2j * math.pi * np.outer(a, a) / nx)


def _to_coeffs(fv: np.ndarray) -> np.ndarray:
    """fhat_k = N^-3 sum_j f(v_j) exp(-i pi k.v_j / L) (inverse of `spectral.to_grid`)."""
    N = fv.shape[0]
    k = spectral.signed(N)
    sgn = np.where(k % 2 == 0, 1.0, -1.0)
    s3 = sgn[:, None, None] * sgn[None, :, None] * sgn[None, None, :]
    return spectral.dft3(fv, -1) * s3 / N ** 3


def transport(fcells: np.ndarray, L: float, Lx: float, t: float) -> np.ndarray:
    """fcells: [n_x][N][N][N] coefficients; returns the cells after free streaming for time t."""
    fcells = np.asarray(fcells, dtype=np.complex128)
    nx, N = fcells.shape[0], fcells.shape[1]
    fv = np.stack([spectral.to_grid(fcells[c], L) for c in range(nx)])           # f(x_c, v_j)
    v1 = -L + 2.0 * L * np.arange(N) / N
    kappa = spectral.signed(nx).astype(np.float64)
    gx = np.einsum("ab,bijk->aijk", _x_dft_matrix(nx, -1), fv)                      # x-DFT
    gx = gx * np.exp(-2j * math.pi * np.outer(kappa, v1) * t / Lx)[:, :, None, None]
    fv = np.einsum("ab,bijk->aijk", _x_dft_matrix(nx, +1), gx) / nx                 # inverse
    return np.stack([_to_coeffs(fv[c]) for c in range(nx)])


def strang(plan: spectral.OraclePlan, fcells: np.ndarray, Lx: float, dt: float, nsteps: int,
           real: bool = False) -> np.ndarray:
    """real: the collision step uses the real-data reading (`spectral.rk4_real`)."""
    rk = spectral.rk4_real if real else spectral.rk4
    f = np.asarray(fcells, dtype=np.complex128).copy()
    for _ in range(nsteps):
        f = transport(f, plan.L, Lx, 0.5 * dt)
        f = np.stack([rk(plan, f[c], dt, 1) for c in range(f.shape[0])])
        f = transport(f, plan.L, Lx, 0.5 * dt)
    return f


def density(fcells: np.ndarray, L: float) -> np.ndarray:
    """rho(x_c) = int f dv = (2L)^3 Re fhat_0 per cell."""
    return (2.0 * L) ** 3 * np.real(np.asarray(fcells)[:, 0, 0, 0])
