"""Angular collision kernels b(cos theta) and their constants.  Oracle: test infrastructure.

All kernels are described by g(theta) = sin(theta) b(cos theta) on (0, pi].

* ``family`` (parameter s in [0, 1)): g = c_s sin^(-1-2s)(theta/2), so that
  g ~ theta^(-1-nu) with nu = 2s (Sec. 2.1, eq. bb).  c_s is fixed by
  lambda = 1/6 (Sec. 5.1, eq. KK3), lambda = (pi/2) int_0^pi sin^2(theta) g dtheta,
  which gives c_s = 1 / (12 pi B(1-s, 3/2)).  s = 0 is the paper's b6 and
  s = 1/2 its b7 (eqs. b6, b7).
* ``b5``: the cutoff kernel b = 1/(4 pi) (eq. b5).
* ``b8``: b = 5 cos(theta/2) / (192 pi sin(theta) sin^(5/2)(theta/2)) (eq. b8).
* ``debye``: g = |log(2 sin(theta/2))| / (2 sin(theta/2)), the angular part of the
  Debye-Yukawa kernel (Sec. 5.4, eq. ApproximatedDebye; its |v - v*| factor is Phi = |q|).
* ``theta0 > 0``: the kernel set to zero for theta < theta0 (eqs. ApproximatedDebyecutoff,
  b3cutoff); there is then no Taylor part and part II starts at theta0.

Part I of the split of Sec. 4.1 needs three moments over [0, eps]:
A1 = int g (1 - cos), A2 = int g (1 - cos)^2, A3 = int g sin^2.
They are evaluated exactly (power series in sin(eps/2) or closed forms).
"""
from __future__ import annotations

import math
from dataclasses import dataclass


def beta_fn(a: float, b: float) -> float:
    return math.exp(math.lgamma(a) + math.lgamma(b) - math.lgamma(a + b))


@dataclass(frozen=True)
class Kernel:
    name: str          # "family", "b5", "b8", "debye"
    s: float = 0.0     # family parameter (nu = 2 s)
    theta0: float = 0.0   # angular cutoff (0: none)

    @property
    def c(self) -> float:
        if self.name == "family":
            return 1.0 / (12.0 * math.pi * beta_fn(1.0 - self.s, 1.5))
        if self.name == "b5":
            return 1.0 / (4.0 * math.pi)
        if self.name == "b8":
            return 5.0 / (192.0 * math.pi)
        if self.name == "debye":
            return 1.0
        raise ValueError(self.name)

    @property
    def kid(self) -> int:
        return {"family": 0, "b5": 1, "b8": 2, "debye": 7}[self.name]

    def g(self, theta):
        """sin(theta) * b(cos theta)."""
        import numpy as np
        th = np.asarray(theta, dtype=np.float64)
        h = np.sin(0.5 * th)
        if self.name == "family":
            return self.c * h ** (-1.0 - 2.0 * self.s)
        if self.name == "b5":
            return self.c * np.sin(th)
        if self.name == "debye":
            return np.abs(np.log(2.0 * h)) / (2.0 * h)
        return self.c * np.cos(0.5 * th) * h ** (-2.5)

    def taylor_moments(self, eps: float):
        """(A1, A2, A3) over [0, eps] (Sec. 4.1, part I after Taylor expansion)."""
        if self.theta0 > 0.0:
            return 0.0, 0.0, 0.0
        W = math.sin(0.5 * eps)
        if self.name == "debye":
            # g (1 - cos) = h |log 2h|, g (1 - cos)^2 = 2 h^3 |log 2h| with h = sin(t/2): no closed
            # form; adaptive quadrature with the logarithmic end weight (library routine)
            # (library routine).  On [0, eps], |log 2h| = -log t - log(2h / t): the first part with
            # QUADPACK's log end weight, the second (smooth, ~ t^2/24) by 16-point Gauss-Legendre.
            import numpy as np
            from scipy.integrate import quad
            from .quadrature import gauss_legendre
            x, w = gauss_legendre(16, 0.0, eps)
            hx = np.sin(0.5 * x)
            corr = -np.log(2.0 * hx / x)
            A1 = -quad(lambda t: math.sin(0.5 * t), 0.0, eps, weight="alg-loga", wvar=(0.0, 0.0))[0] \
                + float(np.sum(w * hx * corr))
            A2 = -quad(lambda t: 2.0 * math.sin(0.5 * t) ** 3, 0.0, eps, weight="alg-loga", wvar=(0.0, 0.0))[0] \
                + float(np.sum(w * 2.0 * hx ** 3 * corr))
            return A1, A2, 2.0 * A1 - A2
        if self.name == "family":
            def int_sin_pow(alpha):
                # int_0^eps sin^alpha(theta/2) dtheta = 2 int_0^asin(W) sin^alpha u du
                #   = 2 sum_n binom(2n, n) 4^-n W^(alpha + 2n + 1) / (alpha + 2n + 1)
                tot, coef, n = 0.0, 1.0, 0
                while True:
                    term = coef * W ** (alpha + 2 * n + 1) / (alpha + 2 * n + 1)
                    tot += term
                    if abs(term) < 1e-30 * abs(tot) or n > 60:
                        break
                    n += 1
                    coef *= (2 * n - 1) / (2 * n)
                return 2.0 * tot
            c = self.c
            A1 = 2.0 * c * int_sin_pow(1.0 - 2.0 * self.s)
            A2 = 4.0 * c * int_sin_pow(3.0 - 2.0 * self.s)
        elif self.name == "b5":
            omc = 2.0 * W * W  # 1 - cos(eps)
            A1 = self.c * omc ** 2 / 2.0
            A2 = self.c * omc ** 3 / 3.0
        else:
            K = self.c
            A1 = 8.0 * K * W ** 0.5
            A2 = 8.0 * K * 0.4 * W ** 2.5
        A3 = 2.0 * A1 - A2  # sin^2 = 2 (1 - cos) - (1 - cos)^2
        return A1, A2, A3

    def lam(self) -> float:
        """lambda = (1/4) int_S2 (1 - (sigma.qhat)^2) b dsigma (Sec. 5.1) by closed form."""
        if self.name == "family":
            return 2.0 * math.pi * self.c * beta_fn(1.0 - self.s, 1.5)
        if self.name == "b5":
            return (math.pi / 2.0) * self.c * 4.0 / 3.0
        return 2.0 * math.pi * self.c * beta_fn(0.25, 2.0)


def kernel_from(name: str, s: float = 0.0) -> Kernel:
    return Kernel(name, float(s))


# ---------------------------------------------------------------------------
# 2D kernels (Sec. 5.2, eqs. b1-b4): b(cos theta) on theta in [0, 2 pi], the measure on S^1
# being d theta; all four give lambda = 1/8 (eq. KK2).  On (0, pi], b = c sin^beta(theta/2)
# (times |cos(theta/2)| for b4).
# ---------------------------------------------------------------------------

_B2D = {  # name: (kid, c, beta, has_cos)
    "b1": (3, 1.0 / (2.0 * math.pi), 0.0, False),
    "b2": (4, 3.0 / 32.0, -1.0, False),
    "b3": (5, 1.0 / (8.0 * math.pi), -2.0, False),
    "b4": (6, 5.0 / 256.0, -2.5, True),
}


def _int_sin_pow(alpha: float, W: float) -> float:
    """int_0^eps sin^alpha(theta/2) d theta, W = sin(eps/2), by the power series of arcsin."""
    tot, coef, n = 0.0, 1.0, 0
    while True:
        term = coef * W ** (alpha + 2 * n + 1) / (alpha + 2 * n + 1)
        tot += term
        if abs(term) < 1e-30 * abs(tot) or n > 60:
            break
        n += 1
        coef *= (2 * n - 1) / (2 * n)
    return 2.0 * tot


@dataclass(frozen=True)
class Kernel2D:
    name: str          # "b1", "b2", "b3", "b4"
    theta0: float = 0.0   # angular cutoff (0: none), eq. b3cutoff

    @property
    def kid(self) -> int:
        return _B2D[self.name][0]

    @property
    def c(self) -> float:
        return _B2D[self.name][1]

    def b(self, theta):
        """b(cos theta) for theta in (0, 2 pi)."""
        import numpy as np
        th = np.asarray(theta, dtype=np.float64)
        _, c, beta, has_cos = _B2D[self.name]
        v = c * np.sin(0.5 * th) ** beta
        return v * np.abs(np.cos(0.5 * th)) if has_cos else v

    def taylor_moments(self, eps: float):
        """(A1, A2, A3) = int_0^eps b (1-cos, (1-cos)^2, sin^2) d theta (parts I and III)."""
        if self.theta0 > 0.0:
            return 0.0, 0.0, 0.0
        _, c, beta, has_cos = _B2D[self.name]
        W = math.sin(0.5 * eps)
        if has_cos:
            # int_0^eps sin^a(t/2) cos(t/2) dt = 2 W^(a+1) / (a+1)
            A1 = 2.0 * c * 2.0 * W ** (beta + 3.0) / (beta + 3.0)
            A2 = 4.0 * c * 2.0 * W ** (beta + 5.0) / (beta + 5.0)
        else:
            A1 = 2.0 * c * _int_sin_pow(beta + 2.0, W)     # 1 - cos = 2 sin^2(t/2)
            A2 = 4.0 * c * _int_sin_pow(beta + 4.0, W)
        A3 = 2.0 * A1 - A2                                  # sin^2 = 2 (1 - cos) - (1 - cos)^2
        return A1, A2, A3

    def lam(self) -> float:
        """lambda = (1/4) int_0^{2 pi} sin^2(theta) b d theta (Sec. 5.1) in closed form: with
        sin^2 = 4 sin^2(t/2) cos^2(t/2) and u = sin(t/2) each kernel is a Beta integral,
        2 c B((beta + 3)/2, (3 + [cos factor])/2)."""
        _, c, beta, has_cos = _B2D[self.name]
        e = 1.0 if has_cos else 0.0
        return 2.0 * c * beta_fn((beta + 3.0) / 2.0, (3.0 + e) / 2.0)
