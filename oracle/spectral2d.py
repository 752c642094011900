"""The 2D spectral collision operator in FP64 (Sec. 2 and Sec. 4 with d = 2).  Oracle: test
infrastructure.

Definitions followed (N modes per axis, signed k in {-N/2, ..., N/2-1}, arrays [N, N]):

* Sec. 4, eq. realQ with d = 2: Qhat_k = sum_p c_p F(k, r_i, qhat_j) sum_{l+m=k} f_l
  (beta_p(m) f_m), c_p = w_i w_j Phi(r_i) r_i^(d-1) (eq. approxG), Phi(r) = r^gamma,
  beta_p(m) = exp(-i pi r_i m.qhat_j / L).  Terms p = i*M + j.
* Quadrature (Sec. 5.2, Table 1): Gauss-Legendre in |q| on [0, R] and the midpoint rule on the
  circle, qhat_j = (cos phi_j, sin phi_j), phi_j = 2 pi (j + 1/2) / M, w_j = 2 pi / M.
* F by the three-part split of Sec. 4.1 (2D case), `ftable.ftable2d`.
* The inner sum as the fast method evaluates it: h = IDFT(f), g_p = IDFT(beta_p f),
  Uhat = DFT(h g_p) / N^2 (circular convolution), the DFT written out per axis.
* `direct_sum2d`: the weighted double sum of eq. sum with G(l, m) = sum_p alpha_p(l+m)
  beta_p(m) (eq. GG1), O(N^4 P), for small N.
* BKW (Sec. 5.1, eqs. BKW and QQ with d = 2; benchmark values C = 1/2, lambda = 1/8, eq. KK2).
"""
from __future__ import annotations

import math

import numpy as np

from . import quadrature
from .ftable import EPS_DEFAULT, ftable2d
from .kernels import Kernel2D
from .spectral import dft_matrix, rk4_steps, signed


def dft2(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised 2D DFT y[j] = sum_k x[k] exp(sign 2 pi i k.j / N), axis by axis."""
    W = dft_matrix(x.shape[0], sign)
    return W @ x @ W.T


def circle_rule(M: int):
    """Midpoint rule on S^1: unit vectors (cos phi_j, sin phi_j), phi_j = 2 pi (j + 1/2) / M."""
    phi = 2.0 * math.pi * (np.arange(M) + 0.5) / M
    return np.stack([np.cos(phi), np.sin(phi)], axis=1), np.full(M, 2.0 * math.pi / M)


class OraclePlan2D:
    """Terms, c_p and the F table of one 2D operator."""

    def __init__(self, N: int, L: float, R: float, gamma: float, kernel: Kernel2D, N_rho: int,
                 M: int, eps: float = EPS_DEFAULT, with_table: bool = True):
        self.N, self.L, self.R, self.gamma, self.kernel = N, L, R, gamma, kernel
        r_i, w_i = quadrature.radial_rule(N_rho, R)
        q_j, w_j = circle_rule(M)
        self.P = N_rho * M
        self.r = np.repeat(r_i, M)
        self.q = np.tile(q_j, (N_rho, 1))
        # c_p = w_r w_q Phi(r) r^(d-1), d = 2
        self.c = np.repeat(w_i, M) * np.tile(w_j, N_rho) * self.r ** gamma * self.r
        self.F = ftable2d(N, L, self.r, self.q, kernel, eps) if with_table else None

    def beta(self, p: int) -> np.ndarray:
        m = signed(self.N).astype(np.float64)
        b1 = np.exp(-1j * math.pi * self.r[p] * m * self.q[p, 0] / self.L)
        b2 = np.exp(-1j * math.pi * self.r[p] * m * self.q[p, 1] / self.L)
        return b1[:, None] * b2[None, :]

    def alpha(self, p: int) -> np.ndarray:
        return self.c[p] * self.F[p]


def collide2d(plan: OraclePlan2D, fhat: np.ndarray, p0: int = 0, p1: int | None = None) -> np.ndarray:
    """Qhat by eq. realQ (d = 2) restricted to terms p0 <= p < p1."""
    N = plan.N
    p1 = plan.P if p1 is None else p1
    fhat = np.asarray(fhat, dtype=np.complex128)
    h = dft2(fhat, +1)
    Q = np.zeros((N, N), dtype=np.complex128)
    for p in range(p0, p1):
        g = dft2(fhat * plan.beta(p), +1)
        Q += plan.alpha(p) * dft2(h * g, -1) / N ** 2
    return Q


def direct_sum2d(plan: OraclePlan2D, fhat: np.ndarray) -> np.ndarray:
    """Eq. sum with the low-rank weight, l = (k - m) mod N, alpha at the output k."""
    N = plan.N
    ks = signed(N)
    K = np.stack(np.meshgrid(ks, ks, indexing="ij"), -1).reshape(-1, 2)
    fl = np.asarray(fhat, dtype=np.complex128).reshape(-1)
    alphas = np.stack([plan.alpha(p).reshape(-1) for p in range(plan.P)])
    betas = np.stack([plan.beta(p).reshape(-1) for p in range(plan.P)])
    Q = np.zeros(N * N, dtype=np.complex128)
    for kk in range(N * N):
        lidx = np.mod(K[kk][None, :] - K, N)
        lflat = lidx[:, 0] * N + lidx[:, 1]
        Gsum = (alphas[:, kk][:, None] * betas).sum(axis=0)
        Q[kk] = np.sum(Gsum * fl * fl[lflat])
    return Q.reshape(N, N)


def eval2d(fhat: np.ndarray, L: float, v: np.ndarray) -> np.ndarray:
    """sum_k fhat_k exp(i pi k.v / L) on the tensor grid v x v (any nodes)."""
    E = np.exp(1j * math.pi * np.outer(v, signed(fhat.shape[0])) / L)
    return E @ fhat @ E.T


def bkw2d_f(v2: np.ndarray, K: float) -> np.ndarray:
    """Eq. BKW with d = 2: (2 pi K)^-1 exp(-|v|^2/2K) ((4K - 2)/(2K) + (1 - K)|v|^2/(2K^2))."""
    return np.exp(-v2 / (2 * K)) / (2 * math.pi * K) * ((4 * K - 2) / (2 * K) + (1 - K) / (2 * K * K) * v2)


def bkw2d_Q(v2: np.ndarray, K: float, lam: float = 0.125) -> np.ndarray:
    """Eq. QQ with d = 2: (2 pi K)^-1 exp(-|v|^2/2K) (1-K)^2 lam / (4 K^4) (8 K^2 - 8 K|v|^2 + |v|^4)."""
    return np.exp(-v2 / (2 * K)) / (2 * math.pi * K) * (1 - K) ** 2 / (4 * K ** 4) * lam * \
        (8 * K * K - 8 * K * v2 + v2 * v2)


def rk4_2d(plan: OraclePlan2D, fhat: np.ndarray, dt: float, nsteps: int) -> np.ndarray:
    """Classical RK4 (Sec. 5.2) on d fhat/dt = collide2d(fhat) (`spectral.rk4_steps`)."""
    return rk4_steps(lambda f: collide2d(plan, f), fhat, dt, nsteps)
