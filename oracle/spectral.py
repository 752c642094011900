"""The spectral collision operator in FP64 (Sec. 2 and Sec. 4).  Oracle: test infrastructure.

Definitions followed (3D, N modes per axis, signed k in {-N/2, ..., N/2-1}):

* Sec. 4, eq. realQ: Qhat_k = sum_p c_p F(k, r_i, qhat_j) sum_{l+m=k} f_l (beta_p(m) f_m),
  c_p = w_i w_j Phi(r_i) r_i^2, Phi(r) = r^gamma (Sec. 1, eq. Bb), and
  beta_p(m) = exp(-i pi r_i m.qhat_j / L).  Terms p = i*M + j.
* The inner sum is evaluated the way the fast method does (Sec. 4: "a few FFTs"):
  h = IDFT(f), g_p = IDFT(beta_p f), Uhat = DFT(h g_p) / N^3 -- a circular
  convolution, l + m = k modulo N.  Here the DFT is written out by definition as a
  matrix along each axis (`dft3`); no FFT library is used.
* `direct_sum`: the same operator as the weighted double sum of eq. sum with the
  low-rank weight of eq. GG1/approxG, summed over pairs (l, m) -- O(N^6 P), small N.
* `padded=True` keeps l + m = k without wrap-around (the literal Galerkin sum of
  eq. sum): DFTs of size 2N, modes outside the N-range zero.
* `collide_real`: f is a real function (Sec. 2), so only the Hermitian part of fhat is data;
  the reading applies eq. realQ to that part with the Nyquist planes (a signed index -N/2,
  which has no partner +N/2 on the grid) set to zero.
"""
from __future__ import annotations

import math

import numpy as np

from . import quadrature
from .ftable import EPS_DEFAULT, ftable
from .kernels import Kernel


def signed(N: int) -> np.ndarray:
    i = np.arange(N)
    return np.where(i < N // 2, i, i - N)


def dft_matrix(N: int, sign: int) -> np.ndarray:
    """W[a, b] = exp(sign 2 pi i a b / N) (definition of the DFT)."""
    a = np.arange(N)
    return np.exp(sign * 2j * math.pi * np.outer(a, a) / N)


def dft3(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised 3D DFT y[j] = sum_k x[k] exp(sign 2 pi i k.j / N), axis by axis: the DFT
    matrix W applied along axis 1, then axis 2, then axis 3 (each a matrix product)."""
    N = x.shape[0]
    W = dft_matrix(N, sign)
    y = (W @ x.reshape(N, N * N)).reshape(N, N, N)           # axis 1: y[a,c,d] = sum_b W[a,b] x[b,c,d]
    y = np.matmul(W[None], y)                                 # axis 2: y[a,c,d] = sum_b W[c,b] y[a,b,d]
    y = (y.reshape(N * N, N) @ W.T).reshape(N, N, N)          # axis 3: y[a,c,d] = sum_b y[a,c,b] W[d,b]
    return y


class OraclePlan:
    """Quadrature terms, c_p, F table and twiddles for one operator (Sec. 4, eq. approxG)."""

    def __init__(self, N: int, L: float, R: float, gamma: float, kernel: Kernel,
                 N_rho: int, M: int, eps: float = EPS_DEFAULT, sphere=None,
                 with_table: bool = True, terms=None):
        self.N, self.L, self.R, self.gamma = N, L, R, gamma
        self.kernel, self.N_rho, self.M, self.eps = kernel, N_rho, M, eps
        r, wr, q, wq = quadrature.terms(N_rho, R, M, sphere)
        self.r, self.wr, self.q, self.wq = r, wr, q, wq
        self.P = len(r)
        # c_p = w_r w_q Phi(r) r^(d-1), d = 3 (eq. approxG)
        self.c = wr * wq * r ** gamma * r ** 2
        self.sel = np.arange(self.P) if terms is None else np.asarray(terms)
        self.F = ftable(N, L, r[self.sel], q[self.sel], kernel, eps) if with_table else None

    def beta_axes(self, p: int):
        """beta_p(m) = prod_d exp(-i pi r m_d qhat_d / L), returned per axis."""
        m = signed(self.N).astype(np.float64)
        return [np.exp(-1j * math.pi * self.r[p] * m * self.q[p, d] / self.L) for d in range(3)]

    def beta(self, p: int) -> np.ndarray:
        b1, b2, b3 = self.beta_axes(p)
        return b1[:, None, None] * b2[None, :, None] * b3[None, None, :]

    def alpha(self, p: int) -> np.ndarray:
        """alpha_p(k) = c_p F(k, r_i, qhat_j) (eq. GG1 with the quadrature of eq. approxG)."""
        idx = int(np.nonzero(self.sel == p)[0][0])
        return self.c[p] * self.F[idx]


def collide(plan: OraclePlan, fhat: np.ndarray, p0: int = 0, p1: int | None = None,
            padded: bool = False) -> np.ndarray:
    """Qhat by eq. realQ restricted to terms p0 <= p < p1 (all terms by default)."""
    N = plan.N
    p1 = plan.P if p1 is None else p1
    fhat = np.asarray(fhat, dtype=np.complex128)
    if padded:
        return _collide_padded(plan, fhat, p0, p1)
    h = dft3(fhat, +1)
    Q = np.zeros((N, N, N), dtype=np.complex128)
    for p in range(p0, p1):
        g = dft3(fhat * plan.beta(p), +1)
        U = dft3(h * g, -1) / N ** 3
        Q += plan.alpha(p) * U
    return Q


def collide_at(plan: OraclePlan, fhat: np.ndarray, kidx, F_at: np.ndarray, p0: int = 0,
               p1: int | None = None) -> np.ndarray:
    """Qhat of eq. realQ over the terms p0 <= p < p1 of `plan` (all by default), at the modes
    kidx[S, 3] (array indices, FFT-natural order) only, with F_at[S, p1 - p0] =
    F(k_s, r_p, qhat_p) supplied by the caller (for example `ftable.fentries`), so a full-size
    operator can be checked at a few modes without the whole F table.  Per term the same steps
    as `collide`: g_p = IDFT(beta_p f) on the whole grid, then the forward DFT of h g_p / N^3
    evaluated at the requested modes only."""
    N = plan.N
    p1 = plan.P if p1 is None else p1
    fhat = np.asarray(fhat, dtype=np.complex128)
    kidx = np.asarray(kidx).reshape(-1, 3)
    v = np.arange(N)
    E = [np.exp(-2j * math.pi * np.outer(kidx[:, d], v) / N) for d in range(3)]     # [S, N] per axis
    h = dft3(fhat, +1)
    Q = np.zeros(len(kidx), dtype=np.complex128)
    for p in range(p0, p1):
        u = h * dft3(fhat * plan.beta(p), +1)
        t = (E[0] @ u.reshape(N, N * N)).reshape(-1, N, N)         # sum over v1
        t = np.einsum("sb,sbc->sc", E[1], t)                        # sum over v2
        U = np.einsum("sc,sc->s", E[2], t) / N ** 3                 # sum over v3
        Q += plan.c[p] * F_at[:, p - p0] * U
    return Q


def nyquist_mask(N: int) -> np.ndarray:
    """True at every mode with a signed index -N/2 on some axis (the Nyquist planes)."""
    ny = signed(N) == -(N // 2)
    return ny[:, None, None] | ny[None, :, None] | ny[None, None, :]


def mirror(x: np.ndarray) -> np.ndarray:
    """y[k] = x[-k], indices modulo N on every axis."""
    N = x.shape[0]
    m = (-np.arange(N)) % N
    return x[np.ix_(m, m, m)]


def real_band(fhat: np.ndarray) -> np.ndarray:
    """Coefficients of the real part of f (Sec. 2: f real means fhat_{-k} = conj fhat_k),
    (fhat_k + conj fhat_{-k}) / 2, with the Nyquist planes set to zero."""
    fhat = np.asarray(fhat, dtype=np.complex128)
    out = 0.5 * (fhat + np.conj(mirror(fhat)))
    out[nyquist_mask(fhat.shape[0])] = 0.0
    return out


def collide_real(plan: OraclePlan, fhat: np.ndarray, p0: int = 0, p1: int | None = None) -> np.ndarray:
    """Real-data reading of eq. realQ: the operator of the real, Nyquist-free part of f
    (`real_band`), every output mode kept."""
    return collide(plan, real_band(fhat), p0, p1)


def rk4_real(plan: OraclePlan, fhat: np.ndarray, dt: float, nsteps: int) -> np.ndarray:
    """Classical RK4 (Sec. 5.2) on d fhat/dt = collide_real(fhat) (`rk4_steps`)."""
    return rk4_steps(lambda f: collide_real(plan, f), fhat, dt, nsteps)


def _embed(x: np.ndarray, N2: int) -> np.ndarray:
    """Place signed modes of an N-grid into an N2-grid (zero elsewhere)."""
    N = x.shape[0]
    k = signed(N) % N2
    out = np.zeros((N2, N2, N2), dtype=np.complex128)
    out[np.ix_(k, k, k)] = x
    return out


def _extract(y: np.ndarray, N: int) -> np.ndarray:
    N2 = y.shape[0]
    k = signed(N) % N2
    return y[np.ix_(k, k, k)]


def _collide_padded(plan, fhat, p0, p1):
    """l + m = k with no wrap-around: DFTs of size 2N so that |l + m| <= N never aliases."""
    N = plan.N
    N2 = 2 * N
    h = dft3(_embed(fhat, N2), +1)
    Q = np.zeros((N, N, N), dtype=np.complex128)
    for p in range(p0, p1):
        g = dft3(_embed(fhat * plan.beta(p), N2), +1)
        U = _extract(dft3(h * g, -1), N) / N2 ** 3
        Q += plan.alpha(p) * U
    return Q


def direct_sum(plan: OraclePlan, fhat: np.ndarray, padded: bool = False) -> np.ndarray:
    """Eq. sum with G(l, m) = sum_p alpha_p(l+m) beta_p(m): a double sum over (l, m).

    Circular form: l = (k - m) mod N, alpha at the output k; padded form: only pairs
    with l + m = k inside the signed range.  O(N^6 P); for N <= 8.
    """
    N = plan.N
    ks = signed(N)
    fl = fhat.reshape(-1)
    K = np.stack(np.meshgrid(ks, ks, ks, indexing="ij"), -1).reshape(-1, 3)
    Q = np.zeros(N ** 3, dtype=np.complex128)
    alphas = np.stack([plan.alpha(p).reshape(-1) for p in range(plan.P)])   # [P, N^3]
    betas = np.stack([plan.beta(p).reshape(-1) for p in range(plan.P)])     # [P, N^3]
    for kk in range(N ** 3):
        kv = K[kk]
        lv = kv[None, :] - K                     # l = k - m for every m
        if padded:
            ok = np.all((lv >= -N // 2) & (lv <= N // 2 - 1), axis=1)
        else:
            ok = np.ones(N ** 3, dtype=bool)
        lidx = np.mod(lv, N)
        lflat = (lidx[:, 0] * N + lidx[:, 1]) * N + lidx[:, 2]
        G = alphas[:, kk][:, None] * betas           # [P, m]
        Gsum = G.sum(axis=0)
        Q[kk] = np.sum((Gsum * fl * fl[lflat])[ok])
    return Q.reshape(N, N, N)


# ---------------------------------------------------------------------------
# Grid values, moments, BKW (Sec. 1 and Sec. 5.1)
# ---------------------------------------------------------------------------

def to_grid(fhat: np.ndarray, L: float) -> np.ndarray:
    """f_N(v_j) = sum_k fhat_k exp(i pi k.v_j / L), v_j = -L + 2 L j / N."""
    N = fhat.shape[0]
    k = signed(N)
    sgn = np.where(k % 2 == 0, 1.0, -1.0)          # exp(-i pi k) from the origin at -L
    s3 = sgn[:, None, None] * sgn[None, :, None] * sgn[None, None, :]
    return dft3(fhat * s3, +1)


def moments(fhat: np.ndarray, L: float) -> np.ndarray:
    """[mass, momentum (3), energy] = int_{D_L} f_N (1, v, |v|^2) dv, exact for the basis.

    int_{-L}^{L} exp(i pi k v / L) dv = 2L delta_k0;
    int v exp(i pi k v/L) dv = (-1)^k 2 L^2 / (i pi k) for k != 0 (0 for k = 0);
    int v^2 exp(i pi k v/L) dv = (-1)^k 4 L^3 / (pi k)^2 for k != 0, 2 L^3 / 3 for k = 0.
    Mass = (2L)^3 Re fhat_0 (Sec. 4, remark on mass).
    """
    N = fhat.shape[0]
    k = signed(N).astype(np.float64)
    sgn = np.where(signed(N) % 2 == 0, 1.0, -1.0)
    I0 = np.where(k == 0, 2 * L, 0.0).astype(np.complex128)
    with np.errstate(divide="ignore", invalid="ignore"):
        I1 = np.where(k == 0, 0.0, sgn * 2 * L * L / (1j * math.pi * k))
        I2 = np.where(k == 0, 2 * L ** 3 / 3.0, sgn * 4 * L ** 3 / (math.pi * k) ** 2)
    I1 = I1.astype(np.complex128)
    I2 = I2.astype(np.complex128)

    def tri(a, b, c):
        return np.einsum("ijk,i,j,k->", fhat, a, b, c)

    mass = tri(I0, I0, I0)
    mom = [tri(I1, I0, I0), tri(I0, I1, I0), tri(I0, I0, I1)]
    energy = tri(I2, I0, I0) + tri(I0, I2, I0) + tri(I0, I0, I2)
    return np.array([mass.real, mom[0].real, mom[1].real, mom[2].real, energy.real])


def bkw_f(v2: np.ndarray, K: float) -> np.ndarray:
    """Eq. BKW in 3D: (2 pi K)^-3/2 exp(-|v|^2/2K) ((5K - 3)/(2K) + (1 - K)|v|^2/(2K^2))."""
    return (2 * math.pi * K) ** -1.5 * np.exp(-v2 / (2 * K)) * \
        ((5 * K - 3) / (2 * K) + (1 - K) / (2 * K * K) * v2)


def bkw_Q(v2: np.ndarray, K: float, lam: float = 1.0 / 6.0) -> np.ndarray:
    """Eq. QQ in 3D: (2 pi K)^-3/2 exp(-|v|^2/2K) (1-K)^2 lam / (4 K^4) (15 K^2 - 10 K|v|^2 + |v|^4)."""
    return (2 * math.pi * K) ** -1.5 * np.exp(-v2 / (2 * K)) * (1 - K) ** 2 / (4 * K ** 4) * lam * \
        (15 * K * K - 10 * K * v2 + v2 * v2)


def grid_v2(N: int, L: float) -> np.ndarray:
    v = -L + 2.0 * L * np.arange(N) / N
    V1, V2, V3 = np.meshgrid(v, v, v, indexing="ij")
    return V1 ** 2 + V2 ** 2 + V3 ** 2


def rk4_steps(rhs, fhat: np.ndarray, dt: float, nsteps: int) -> np.ndarray:
    """Classical fourth-order Runge-Kutta (Sec. 5.2) on d fhat/dt = rhs(fhat): per step the four
    stage slopes k1 = rhs(f), k2 = rhs(f + dt k1 / 2), k3 = rhs(f + dt k2 / 2), k4 = rhs(f + dt k3),
    then f + dt (k1 + 2 k2 + 2 k3 + k4) / 6.  The one stage formula every oracle RK4 uses."""
    f = np.asarray(fhat, dtype=np.complex128).copy()
    for _ in range(nsteps):
        k1 = rhs(f)
        k2 = rhs(f + 0.5 * dt * k1)
        k3 = rhs(f + 0.5 * dt * k2)
        k4 = rhs(f + dt * k3)
        f = f + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return f


def rk4(plan: OraclePlan, fhat: np.ndarray, dt: float, nsteps: int) -> np.ndarray:
    """Classical RK4 (Sec. 5.2) on d fhat/dt = Qhat(fhat) (`rk4_steps`)."""
    return rk4_steps(lambda f: collide(plan, f), fhat, dt, nsteps)
