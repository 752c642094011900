"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the bench.

This module holds no arithmetic of the collision operator.  It draws random
numbers (SplitMix64, Steele, Lea & Flood 2014) and evaluates the Fourier
coefficients of the synthetic velocity distributions used as workloads:

* sums of isotropic or anisotropic Gaussians (closed-form Fourier transform),
* the BKW solution of the Maxwell-molecule problem (Sec. 5.1, eq. BKW),
* a Gaussian plus seeded per-grid-point noise (grid samples, then a library DFT).

Coefficient convention (Sec. 2): f_N(v) = sum_k fhat_k exp(i pi k.v / L) on
[-L, L]^3, fhat_k = (2L)^-3 int f(v) exp(-i pi k.v / L) dv.  Arrays are
complex128, C-order [k1][k2][k3], FFT-natural index order: array index i holds
the signed mode k = i if i < N/2 else i - N.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """SplitMix64 stream; `uniform(n)` returns doubles (x >> 11) * 2^-53 in [0, 1)."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            steps = np.arange(1, n + 1, dtype=np.uint64) * _GOLDEN
            z = self.state + steps
            self.state = self.state + np.uint64(n) * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def signed_modes(N: int) -> np.ndarray:
    """Signed mode index for each FFT-natural array index (length N, even N)."""
    i = np.arange(N)
    return np.where(i < N // 2, i, i - N)


def _omega(N: int, L: float):
    k = signed_modes(N).astype(np.float64)
    w = math.pi * k / L
    return np.meshgrid(w, w, w, indexing="ij")


def gaussian_mixture_fhat(N: int, L: float, masses, centers, temps) -> np.ndarray:
    """Fourier coefficients of sum_g m_g (2 pi T_g)^-3/2 exp(-|v - u_g|^2 / (2 T_g)).

    `temps[g]` may be a scalar (isotropic) or a length-3 sequence (T_x, T_y, T_z).
    The transform is taken over R^3; the mass outside [-L, L]^3 is assumed negligible.
    """
    w1, w2, w3 = _omega(N, L)
    out = np.zeros((N, N, N), dtype=np.complex128)
    for m, u, T in zip(masses, centers, temps):
        T = np.broadcast_to(np.asarray(T, dtype=np.float64), (3,))
        phase = np.exp(-1j * (w1 * u[0] + w2 * u[1] + w3 * u[2]))
        damp = np.exp(-0.5 * (T[0] * w1 ** 2 + T[1] * w2 ** 2 + T[2] * w3 ** 2))
        out += m * phase * damp
    return out / (2.0 * L) ** 3


def bkw_K(t: float, lam: float = 1.0 / 6.0, C: float = 1.0) -> float:
    """K(t) = 1 - C exp(-lambda t) (Sec. 5.1, 3D benchmark values C = 1, lambda = 1/6)."""
    return 1.0 - C * math.exp(-lam * t)


def bkw_fhat(N: int, L: float, K: float) -> np.ndarray:
    """Fourier coefficients of the 3D BKW profile (Sec. 5.1, eq. BKW) at a given K.

    f(v) = (2 pi K)^-3/2 exp(-|v|^2/(2K)) (A + B |v|^2), A = (5K-3)/(2K),
    B = (1-K)/(2K^2); its transform is (A + B (3K - K^2 |w|^2)) exp(-K |w|^2 / 2).
    """
    w1, w2, w3 = _omega(N, L)
    w2sum = w1 ** 2 + w2 ** 2 + w3 ** 2
    A = (5.0 * K - 3.0) / (2.0 * K)
    B = (1.0 - K) / (2.0 * K * K)
    val = (A + B * (3.0 * K - K * K * w2sum)) * np.exp(-0.5 * K * w2sum)
    return val.astype(np.complex128) / (2.0 * L) ** 3


def bkw2d_K(t: float, lam: float = 0.125, C: float = 0.5) -> float:
    """K(t) = 1 - C exp(-lambda t) with the 2D benchmark values C = 1/2, lambda = 1/8 (Sec. 5.1)."""
    return 1.0 - C * math.exp(-lam * t)


def bkw2d_fhat(N: int, L: float, K: float) -> np.ndarray:
    """Fourier coefficients [N, N] of the 2D BKW profile (Sec. 5.1, eq. BKW with d = 2).

    f(v) = (2 pi K)^-1 exp(-|v|^2/(2K)) (A + B |v|^2), A = (2K-1)/K, B = (1-K)/(2K^2); its
    transform is (A + B (2K - K^2 |w|^2)) exp(-K |w|^2 / 2), sampled at w = pi k / L.
    """
    w = math.pi * signed_modes(N).astype(np.float64) / L
    W1, W2 = np.meshgrid(w, w, indexing="ij")
    w2sum = W1 ** 2 + W2 ** 2
    A = (2.0 * K - 1.0) / K
    B = (1.0 - K) / (2.0 * K * K)
    val = (A + B * (2.0 * K - K * K * w2sum)) * np.exp(-0.5 * K * w2sum)
    return val.astype(np.complex128) / (2.0 * L) ** 2


def grid2d_cells(N: int, L: float) -> np.ndarray:
    """Cell-centred 2D velocity nodes v_j = -L + 2L (j + 1/2) / N (the grid of Table 1)."""
    return -L + 2.0 * L * (np.arange(N) + 0.5) / N


def bkw2d_fhat_samples(N: int, L: float, K: float) -> np.ndarray:
    """[N, N] coefficients whose trigonometric interpolant takes the 2D BKW values (Sec. 5.1,
    eq. BKW, d = 2) at the cell-centred nodes: fhat_k = N^-2 sum_j f(v_j) exp(-i pi k.v_j / L)."""
    v = grid2d_cells(N, L)
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    v2 = V1 ** 2 + V2 ** 2
    f = np.exp(-v2 / (2 * K)) / (2 * math.pi * K) * ((4 * K - 2) / (2 * K) + (1 - K) / (2 * K * K) * v2)
    E = np.exp(-1j * math.pi * np.outer(signed_modes(N), v) / L)
    return E @ f @ E.T / N ** 2


def random_mixture2d(N: int, L: float, seed: int, box: float = 2.0) -> np.ndarray:
    """Two 2D Maxwellians of mass 1/2, centres uniform in [-box, box]^2, T in [0.5, 2]."""
    u = SplitMix64(seed).uniform(6)
    w = math.pi * signed_modes(N).astype(np.float64) / L
    W1, W2 = np.meshgrid(w, w, indexing="ij")
    out = np.zeros((N, N), dtype=np.complex128)
    for g in range(2):
        c1, c2 = box * (2 * u[3 * g] - 1), box * (2 * u[3 * g + 1] - 1)
        T = 0.5 + 1.5 * u[3 * g + 2]
        out += 0.5 * np.exp(-1j * (W1 * c1 + W2 * c2) - 0.5 * T * (W1 ** 2 + W2 ** 2))
    return out / (2.0 * L) ** 2


def grid_samples_to_fhat(fv: np.ndarray, L: float) -> np.ndarray:
    """fhat_k = N^-3 sum_j f(v_j) exp(-i pi k.v_j/L) with v_j = -L + 2L j/N (library FFT)."""
    N = fv.shape[0]
    k = signed_modes(N)
    sign = np.where(k % 2 == 0, 1.0, -1.0)  # exp(i pi k) from the grid origin at -L
    s3 = sign[:, None, None] * sign[None, :, None] * sign[None, None, :]
    return np.fft.fftn(fv) / N ** 3 * s3


def grid(N: int, L: float) -> np.ndarray:
    return -L + 2.0 * L * np.arange(N) / N


def _samples_to_fhat(fv: np.ndarray, L: float) -> np.ndarray:
    """fhat_k = N^-d sum_j f(v_j) exp(-i pi k.v_j / L), nodes v_j = -L + 2L j/N, any d (library FFT)."""
    N, d = fv.shape[0], fv.ndim
    sign = np.where(signed_modes(N) % 2 == 0, 1.0, -1.0)
    s = sign
    for _ in range(d - 1):
        s = np.multiply.outer(s, sign)
    return np.fft.fftn(fv) / N ** d * s


def delta_w(x, w: float) -> np.ndarray:
    """Approximate delta (Sec. 5.3, eq. delta): (1 + cos(pi x / w)) / (2w) for |x| <= w, else 0."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(np.abs(x) <= w, (1.0 + np.cos(np.pi * x / w)) / (2.0 * w), 0.0)


def _speed(N: int, L: float, d: int) -> np.ndarray:
    v = grid(N, L)
    V = np.meshgrid(*([v] * d), indexing="ij")
    return np.sqrt(sum(x * x for x in V))


def measure_valued_fhat(N: int, L: float, d: int, rings=((0.0, 1.0 / 3.0), (0.2, 1.0 / 3.0))) -> np.ndarray:
    """Coefficients of f0(v) = sum_r c_r delta_w(|v| - rho_r) on the d-dimensional grid, with
    w = 0.5 sqrt(dv), dv = 2L/N (Sec. 5.3, eq. initialdelta; eq. initialdelta1 is rings =
    ((0.2, 0.5),)), from the grid samples."""
    w = 0.5 * math.sqrt(2.0 * L / N)
    sp = _speed(N, L, d)
    fv = sum(c * delta_w(sp - rho, w) for rho, c in rings)
    return _samples_to_fhat(fv, L)


def discontinuous2d_fhat(N: int, L: float) -> np.ndarray:
    """Coefficients of the 2D discontinuous data of Sec. 5.5 (eq. disinitial): rho_1 / (2 pi T_1)
    exp(-|v|^2 / 2 T_1) for v_1 > 0 and rho_2 / (2 pi T_2) exp(-|v|^2 / 2 T_2) for v_1 < 0, with
    rho = (6/5, 4/5), T = (2/3, 3/2); v_1 = 0 takes the mean.  From the grid samples."""
    v = grid(N, L)
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    v2 = V1 ** 2 + V2 ** 2
    g1 = 1.2 / (2 * math.pi * (2.0 / 3.0)) * np.exp(-v2 / (2 * (2.0 / 3.0)))
    g2 = 0.8 / (2 * math.pi * 1.5) * np.exp(-v2 / (2 * 1.5))
    fv = np.where(V1 > 0, g1, np.where(V1 < 0, g2, 0.5 * (g1 + g2)))
    return _samples_to_fhat(fv, L)


# ---------------------------------------------------------------------------
# Workload recipes (seeded).  Each returns complex128 [N, N, N].
# ---------------------------------------------------------------------------

def two_maxwellians_c1(N: int, L: float) -> np.ndarray:
    """Equal-mass unit-temperature Maxwellians centred at +-2 e1 (total mass 1)."""
    return gaussian_mixture_fhat(N, L, [0.5, 0.5], [(2.0, 0, 0), (-2.0, 0, 0)], [1.0, 1.0])


def bigaussian_noise_c3(N: int, L: float, seed: int = 3) -> np.ndarray:
    """Anisotropic bi-Gaussian (T = 2, 0.5, 0.5, mass 1) plus 0.01 U_j G(v_j), U_j ~ U[0,1).

    G is the unit-temperature Maxwellian; U_j is drawn per grid point in C-order.
    """
    base = gaussian_mixture_fhat(N, L, [1.0], [(0.0, 0.0, 0.0)], [(2.0, 0.5, 0.5)])
    v = grid(N, L)
    V1, V2, V3 = np.meshgrid(v, v, v, indexing="ij")
    G = (2 * math.pi) ** -1.5 * np.exp(-0.5 * (V1 ** 2 + V2 ** 2 + V3 ** 2))
    U = SplitMix64(seed).uniform(N ** 3).reshape(N, N, N)
    return base + grid_samples_to_fhat(0.01 * U * G, L)


def random_mixture(N: int, L: float, seed: int, box: float = 3.0) -> np.ndarray:
    """Two Maxwellians of mass 1/2, centres U[-box, box]^3, temperatures U[0.5, 2]."""
    u = SplitMix64(seed).uniform(8)
    c1 = tuple(-box + 2 * box * u[0:3])
    c2 = tuple(-box + 2 * box * u[3:6])
    T1 = 0.5 + 1.5 * u[6]
    T2 = 0.5 + 1.5 * u[7]
    return gaussian_mixture_fhat(N, L, [0.5, 0.5], [c1, c2], [T1, T2])


def random_fhat(N: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Unstructured complex coefficients with entries U[-1,1) + i U[-1,1) (no symmetry)."""
    u = SplitMix64(seed).uniform(2 * N ** 3)
    re = (2 * u[0::2] - 1).reshape(N, N, N)
    im = (2 * u[1::2] - 1).reshape(N, N, N)
    return scale * (re + 1j * im)


def inhom_cells(N: int, L: float, nx: int, Lx: float, eps: float = 0.2) -> np.ndarray:
    """[nx][N^3] coefficients of f(x_c, v) = (1 + eps cos(2 pi x_c / Lx)) (M(v - u_c e1) + M(v + u_c e1)) / 2,
    x_c = c Lx / nx, u_c = 1 + 0.5 sin(2 pi x_c / Lx), unit-temperature Maxwellians M: a density
    wave on a two-stream velocity profile whose separation varies along x."""
    out = np.empty((nx, N, N, N), dtype=np.complex128)
    for c in range(nx):
        x = c * Lx / nx
        rho = 1.0 + eps * math.cos(2 * math.pi * x / Lx)
        u = 1.0 + 0.5 * math.sin(2 * math.pi * x / Lx)
        out[c] = gaussian_mixture_fhat(N, L, [0.5 * rho, 0.5 * rho], [(u, 0.0, 0.0), (-u, 0.0, 0.0)], [1.0, 1.0])
    return out


def drifting_wave_samples(N: int, L: float, nx: int, Lx: float, eps: float, u: float, T: float) -> np.ndarray:
    """[nx][N^3] coefficients from the node values of f(x_c, v) = (1 + eps cos(2 pi x_c / Lx)) M_T(v - u e1)
    (M_T the Maxwellian of temperature T), taken by the library FFT of the samples."""
    v = grid(N, L)
    V1, V2, V3 = np.meshgrid(v, v, v, indexing="ij")
    M = (2 * math.pi * T) ** -1.5 * np.exp(-((V1 - u) ** 2 + V2 ** 2 + V3 ** 2) / (2 * T))
    out = np.empty((nx, N, N, N), dtype=np.complex128)
    for c in range(nx):
        out[c] = _samples_to_fhat((1.0 + eps * math.cos(2 * math.pi * c / nx)) * M, L)
    return out


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process (exponential gaps from SplitMix64)."""
    u = SplitMix64(seed).uniform(n)
    gaps = -np.log1p(-u) / rate
    return np.cumsum(gaps)


# Domains used by the workloads (Sec. 2: L >= (3 + sqrt 2) S / 2 with R = 2S).
def R_from_L(L: float) -> float:
    return 4.0 * L / (3.0 + math.sqrt(2.0))


def L_from_R(R: float) -> float:
    return (3.0 + math.sqrt(2.0)) * R / 4.0
