"""Quadrature rules for |q| and qhat (Sec. 4, eq. approxG).  Oracle: test infrastructure.

* radial: N_rho-point Gauss-Legendre on [0, R] (the paper's choice),
* sphere: the paper uses Womersley spherical designs, which are not available
  here; this oracle uses the icosahedron for M = 12 (a spherical 5-design with
  equal weights 4 pi / 12) and for other M a product rule: n_t Gauss-Legendre
  points in cos(theta) times n_p equispaced azimuths phi_b = 2 pi (b + 1/2) / n_p,
  with M = n_t * n_p, n_p = 2 n_t when M = 2 n^2, n_p = n_t when M = n^2.
"""
from __future__ import annotations

import math

import numpy as np


def gauss_legendre(n: int, a: float = -1.0, b: float = 1.0):
    """n-point Gauss-Legendre nodes and weights on [a, b] (library routine, mapped)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def radial_rule(N_rho: int, R: float):
    """|q| nodes r_i and weights w_i on [0, R] (Sec. 4: Gauss-Legendre in |q|)."""
    return gauss_legendre(N_rho, 0.0, R)


def icosahedron():
    """12 unit vertices (0, +-1, +-phi) and cyclic permutations, weights 4 pi / 12."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    pts = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            pts.append((0.0, s1, s2 * phi))
            pts.append((s1, s2 * phi, 0.0))
            pts.append((s2 * phi, 0.0, s1))
    P = np.array(pts)
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    return P, np.full(12, 4.0 * math.pi / 12.0)


def product_rule(n_t: int, n_p: int):
    """Gauss-Legendre in cos(theta) (n_t points) times midpoint azimuths (n_p points)."""
    ct, wt = gauss_legendre(n_t)
    st = np.sqrt(1.0 - ct ** 2)
    phi = 2.0 * math.pi * (np.arange(n_p) + 0.5) / n_p
    pts, wts = [], []
    for a in range(n_t):
        for b in range(n_p):
            pts.append((st[a] * math.cos(phi[b]), st[a] * math.sin(phi[b]), ct[a]))
            wts.append(wt[a] * 2.0 * math.pi / n_p)
    return np.array(pts), np.array(wts)


def sphere_rule(M: int):
    """Sphere rule with M points: icosahedron for 12, else the product rule above."""
    if M == 12:
        return icosahedron()
    n = int(round(math.sqrt(M / 2.0)))
    if 2 * n * n == M:
        return product_rule(n, 2 * n)
    n = int(round(math.sqrt(M)))
    if n * n == M:
        return product_rule(n, n)
    raise ValueError(f"no built-in sphere rule with M={M} points")


def terms(N_rho: int, R: float, M: int, sphere=None):
    """Quadrature terms p = i*M + j (radial index i major, sphere index j minor).

    Returns r[P], wr[P], qhat[P,3], wq[P].
    """
    r, wr = radial_rule(N_rho, R)
    q, wq = sphere_rule(M) if sphere is None else sphere
    rr = np.repeat(r, len(wq))
    wrr = np.repeat(wr, len(wq))
    qq = np.tile(q, (N_rho, 1))
    wqq = np.tile(wq, N_rho)
    return rr, wrr, qq, wqq
