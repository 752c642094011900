"""F(k, |q|, qhat) of Sec. 2.1 eq. FF by the split of Sec. 4.1.  Oracle: test infrastructure.

`ftable` / `fentries` call the C code in ftable.c (built by `build()`), which
follows the paper's split: part I by Taylor expansion (exact kernel moments),
part II by a converged composite Gauss-Legendre rule, phi integral exact (J0).

Two further routes exist only to pin the first one:
* `f_exact_series`: the exact F (no Taylor step) by the Funk-Hecke theorem,
  F = exp(i z mu) sum_{l>=1} (2l+1) (-i)^l j_l(z) P_l(mu) (lambda_l - lambda_0),
  z = a|k|, mu = khat.qhat, lambda_l = 2 pi int_{-1}^{1} b(t) P_l(t) dt.
  It differs from the split by the Taylor remainder over [0, eps] only.
* `f_phi_midpoint`: the paper's literal phi midpoint rule in place of J0.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

from .kernels import Kernel
from .quadrature import gauss_legendre

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None

EPS_DEFAULT = math.pi / 1000.0   # Sec. 4.1: epsilon = pi / 1000
NPTS_DEFAULT = 20                # Gauss-Legendre points per panel of part II


def build(force: bool = False) -> str:
    """Compile ftable.c and ftable2d.c into _build/liboracle.so with gcc (FP64, OpenMP)."""
    srcs = [os.path.join(_HERE, "ftable.c"), os.path.join(_HERE, "ftable2d.c")]
    if not force and os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(x) for x in srcs):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
                           "-o", tmp] + srcs + ["-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_ftable.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, dp,
                                      ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, dp, ctypes.c_int, dp, dp, dp]
        lib.oracle_ftable.restype = ctypes.c_int
        lib.oracle_fentries.argtypes = [ctypes.c_int, ip, dp, dp, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, dp, ctypes.c_int, dp, dp, dp]
        lib.oracle_fentries.restype = ctypes.c_int
        lib.oracle_ftable2d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, dp,
                                        ctypes.c_int, ctypes.c_double, ctypes.c_double, dp,
                                        ctypes.c_int, dp, dp, dp]
        lib.oracle_ftable2d.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def ftable(N: int, L: float, r, qhat, kernel: Kernel, eps: float = EPS_DEFAULT,
           npts: int = NPTS_DEFAULT) -> np.ndarray:
    """F for every mode k (signed, FFT-natural order) and term (r[p], qhat[p]); [P, N, N, N] c128."""
    lib = _load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    qhat = np.ascontiguousarray(qhat, dtype=np.float64).reshape(-1, 3)
    P = len(r)
    A = np.array(kernel.taylor_moments(eps), dtype=np.float64)
    gx, gw = gauss_legendre(npts)
    gx = np.ascontiguousarray(gx)
    gw = np.ascontiguousarray(gw)
    out = np.empty((P, N, N, N), dtype=np.complex128)
    lo = kernel.theta0 if kernel.theta0 > 0 else eps     # lower end of part II
    rc = lib.oracle_ftable(N, L, P, _dp(r), _dp(qhat), kernel.kid, kernel.s, kernel.c, lo,
                           _dp(A), npts, _dp(gx), _dp(gw), _dp(out.view(np.float64)))
    if rc != 0:
        raise MemoryError("oracle_ftable failed")
    return out


def fentries(N: int, L: float, k, r, qhat, kernel: Kernel, eps: float = EPS_DEFAULT,
             npts: int = NPTS_DEFAULT) -> np.ndarray:
    """F at individual entries: k[E,3] signed ints, r[E], qhat[E,3]; N sets the part-II rule."""
    lib = _load()
    k = np.ascontiguousarray(k, dtype=np.int32).reshape(-1, 3)
    r = np.ascontiguousarray(r, dtype=np.float64)
    qhat = np.ascontiguousarray(qhat, dtype=np.float64).reshape(-1, 3)
    A = np.array(kernel.taylor_moments(eps), dtype=np.float64)
    gx, gw = gauss_legendre(npts)
    gx = np.ascontiguousarray(gx)
    gw = np.ascontiguousarray(gw)
    out = np.empty(len(r), dtype=np.complex128)
    lo = kernel.theta0 if kernel.theta0 > 0 else eps
    rc = lib.oracle_fentries(len(r), k.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(r),
                             _dp(qhat), L, N, kernel.kid, kernel.s, kernel.c, lo, _dp(A), npts,
                             _dp(gx), _dp(gw), _dp(out.view(np.float64)))
    if rc != 0:
        raise MemoryError("oracle_fentries failed")
    return out


def ftable2d(N: int, L: float, r, qhat, kernel, eps: float = EPS_DEFAULT,
             npts: int = NPTS_DEFAULT) -> np.ndarray:
    """2D F (eq. FF2D1, three-part split of Sec. 4.1) for every mode of the N^2 grid and term
    (r[p], qhat[p] in R^2); [P, N, N] c128.  kernel is a kernels.Kernel2D."""
    lib = _load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    qhat = np.ascontiguousarray(qhat, dtype=np.float64).reshape(-1, 2)
    P = len(r)
    A = np.array(kernel.taylor_moments(eps), dtype=np.float64)
    gx, gw = gauss_legendre(npts)
    gx = np.ascontiguousarray(gx)
    gw = np.ascontiguousarray(gw)
    out = np.empty((P, N, N), dtype=np.complex128)
    lo = kernel.theta0 if kernel.theta0 > 0 else eps
    rc = lib.oracle_ftable2d(N, L, P, _dp(r), _dp(qhat), kernel.kid, kernel.c, lo, _dp(A), npts,
                             _dp(gx), _dp(gw), _dp(out.view(np.float64)))
    if rc != 0:
        raise MemoryError("oracle_ftable2d failed")
    return out


# ---------------------------------------------------------------------------
# Independent routes (pins only)
# ---------------------------------------------------------------------------

def _legendre_minus_one_series(l: int, u, terms: int = 14):
    """P_l(1 - 2u) - 1 = sum_{m>=1} (-1)^m C(l,m) C(l+m,m) u^m (hypergeometric form)."""
    u = np.asarray(u, dtype=np.float64)
    tot = np.zeros_like(u)
    t = np.ones_like(u)
    for m in range(0, min(l, terms)):
        # ratio t_{m+1}/t_m = -(l-m)(l+m+1) u / (m+1)^2
        t = t * (-(l - m) * (l + m + 1) * u / ((m + 1) ** 2))
        tot = tot + t
    return tot


def funk_hecke_eigen(kernel: Kernel, lmax: int) -> np.ndarray:
    """lambda_l - lambda_0 = 2 pi int_0^pi g(t) (P_l(cos t) - 1) dt for l = 0..lmax."""
    from scipy import integrate, special
    out = np.zeros(lmax + 1)
    if kernel.theta0 > 0 or kernel.name == "debye":
        # no algebraic end singularity to weight: g (P_l - 1) is bounded (~ t |log t| for the
        # Debye-Yukawa kernel) or zero near 0; plain adaptive quadrature with the pi/3 kink as a
        # break point
        lo = kernel.theta0
        pts = [p for p in (math.pi / 3.0,) if lo < p]
        for l in range(1, lmax + 1):
            fl = lambda t, l=l: float(kernel.g(max(t, 1e-300))) * (special.eval_legendre(l, math.cos(t)) - 1.0)
            out[l] = 2.0 * math.pi * integrate.quad(fl, lo, math.pi, points=pts or None, epsabs=1e-15,
                                                   epsrel=1e-13, limit=4000)[0]
        return out
    alpha = {"family": 1.0 - 2.0 * kernel.s, "b5": 1.0, "b8": -0.5}[kernel.name]
    for l in range(1, lmax + 1):
        ts = min(0.63 / l, 0.5)

        def f_small(t, l=l):
            t = max(t, 1e-9)      # the quotient is smooth; its value at t -> 0 is the limit
            u = math.sin(0.5 * t) ** 2
            return float(kernel.g(t)) * float(_legendre_minus_one_series(l, u)) / t ** alpha

        def f_big(t, l=l):
            return float(kernel.g(t)) * (special.eval_legendre(l, math.cos(t)) - 1.0)

        a, _ = integrate.quad(f_small, 0.0, ts, weight="alg", wvar=(alpha, 0.0),
                              epsabs=1e-15, epsrel=1e-13, limit=200)
        b, _ = integrate.quad(f_big, ts, math.pi, epsabs=1e-15, epsrel=1e-13,
                              limit=2000)
        out[l] = 2.0 * math.pi * (a + b)
    return out


def f_exact_series(k, r: float, qhat, L: float, kernel: Kernel, eig=None) -> complex:
    """Exact F(k, r, qhat) (no Taylor step) by the Funk-Hecke expansion of the plane wave."""
    from scipy import special
    k = np.asarray(k, dtype=np.float64)
    qhat = np.asarray(qhat, dtype=np.float64)
    a = math.pi * r / (2.0 * L)
    kn = float(np.linalg.norm(k))
    if kn == 0.0:
        return 0.0 + 0.0j
    z = a * kn
    mu = float(k @ qhat) / kn
    lmax = int(z + 40)
    if eig is None or len(eig) <= lmax:
        eig = funk_hecke_eigen(kernel, lmax)
    s = 0.0 + 0.0j
    for l in range(1, lmax + 1):
        s += (2 * l + 1) * (-1j) ** l * special.spherical_jn(l, z) * \
            special.eval_legendre(l, mu) * eig[l]
    return complex(np.exp(1j * z * mu) * s)


def taylor_remainder_bound(z: float, kernel: Kernel, eps: float = EPS_DEFAULT) -> float:
    """Bound on |F_split - F_exact| from the Taylor step on [0, eps].

    With w = i (A - B cos psi), |A| <= z t^2 / 2, |B| <= z t, the phi-averaged
    remainder of exp(w) - 1 - w - w^2/2 is at most (|A|^3 + 1.5 |A| B^2) / 6
    + (|A| + |B|)^4 / 24; integrate 2 pi g(t) times that over [0, eps].
    """
    from scipy import integrate

    def f(t):
        A = 0.5 * z * t * t
        B = z * t
        return float(kernel.g(t)) * ((A ** 3 + 1.5 * A * B * B) / 6.0 + (A + B) ** 4 / 24.0)

    val, _ = integrate.quad(f, 0.0, eps, limit=200)
    return 2.0 * math.pi * val


def f_phi_midpoint(k, r: float, qhat, L: float, kernel: Kernel, nphi: int,
                   eps: float = EPS_DEFAULT, npts: int = 24, width: float = 0.05) -> complex:
    """F by the paper's literal recipe: part I Taylor moments, part II a theta rule times
    the midpoint rule in phi (nphi points) applied to exp(i a k.(qhat - sigma)) - 1."""
    k = np.asarray(k, dtype=np.float64)
    qhat = np.asarray(qhat, dtype=np.float64)
    a = math.pi * r / (2.0 * L)
    kap = float(k @ qhat)
    kperp = k - kap * qhat
    kp = float(np.linalg.norm(kperp))
    A1, A2, A3 = kernel.taylor_moments(eps)
    x, y = a * kap, a * kp
    part1 = 2 * math.pi * (1j * x * A1 - 0.5 * x * x * A2 - 0.25 * y * y * A3)
    edges = [eps]
    while edges[-1] < 0.5:
        edges.append(min(2 * edges[-1], 0.5))
    n_uni = int(math.ceil((math.pi - 0.5) / width))
    edges += list(np.linspace(0.5, math.pi, n_uni + 1)[1:])
    gx, gw = gauss_legendre(npts)
    phi = 2 * math.pi * (np.arange(nphi) + 0.5) / nphi
    part2 = 0.0 + 0.0j
    for lo, hi in zip(edges[:-1], edges[1:]):
        t = 0.5 * (hi - lo) * gx + 0.5 * (hi + lo)
        w = 0.5 * (hi - lo) * gw * kernel.g(t)
        # k.(qhat - sigma) = kappa (1 - cos t) - kperp sin t cos phi
        arg = x * (1 - np.cos(t))[:, None] - y * np.sin(t)[:, None] * np.cos(phi)[None, :]
        inner = (np.exp(1j * arg) - 1.0).mean(axis=1) * 2 * math.pi
        part2 += np.sum(w * inner)
    return complex(part1 + part2)
