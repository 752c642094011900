"""Pins for the oracle's quadrature rules and kernel constants (CPU only)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import kernels, quadrature


def _sphere_monomial(a, b, c):
    """int_{S^2} x^a y^b z^c dsigma (0 unless all even) = 2 G(A)G(B)G(C)/G(A+B+C), A=(a+1)/2."""
    if a % 2 or b % 2 or c % 2:
        return 0.0
    A, B, C = (a + 1) / 2, (b + 1) / 2, (c + 1) / 2
    return 2 * math.gamma(A) * math.gamma(B) * math.gamma(C) / math.gamma(A + B + C)


@pytest.mark.parametrize("n", [1, 4, 16, 32])
def test_radial_gauss_legendre_exact_to_degree_2n_minus_1(n):
    R = 6.0
    r, w = quadrature.radial_rule(n, R)
    for d in range(2 * n):
        exact = R ** (d + 1) / (d + 1)
        assert abs(np.sum(w * r ** d) - exact) <= 1e-13 * exact
    if n <= 4:    # not exact one degree higher (guards against a rule of the wrong size)
        d = 2 * n
        assert abs(np.sum(w * r ** d) - R ** (d + 1) / (d + 1)) > 1e-10 * R ** (d + 1) / (d + 1)


def _max_monomial_error(P, w, deg):
    err = 0.0
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                val = np.sum(w * P[:, 0] ** a * P[:, 1] ** b * P[:, 2] ** c)
                err = max(err, abs(val - _sphere_monomial(a, b, c)))
    return err


def test_icosahedron_is_a_5_design():
    P, w = quadrature.icosahedron()
    assert np.allclose(np.linalg.norm(P, axis=1), 1.0, atol=1e-15)
    assert _max_monomial_error(P, w, 5) < 1e-13
    # degree 6 is not integrated exactly
    assert abs(np.sum(w * P[:, 2] ** 6) - _sphere_monomial(0, 0, 6)) > 1e-4


@pytest.mark.parametrize("M,deg", [(32, 7), (64, 7), (72, 11)])
def test_product_rule_exactness(M, deg):
    P, w = quadrature.sphere_rule(M)
    assert len(w) == M
    assert abs(np.sum(w) - 4 * math.pi) < 1e-13
    assert _max_monomial_error(P, w, deg) < 1e-12


@pytest.mark.parametrize("name,s,paper_c", [
    ("family", 0.0, 1.0 / (8 * math.pi)),          # eq. b6
    ("family", 0.5, 1.0 / (6 * math.pi ** 2)),     # eq. b7
    ("family", 0.25, None), ("family", 0.75, None),
    ("b5", 0.0, 1.0 / (4 * math.pi)),              # eq. b5
    ("b8", 0.0, 5.0 / (192 * math.pi)),            # eq. b8
])
def test_kernel_lambda_is_one_sixth(name, s, paper_c):
    """Sec. 5.1: lambda = (1/4) int (1 - (sigma.qhat)^2) b dsigma = 1/6 for every 3D kernel."""
    k = kernels.Kernel(name, s)
    if paper_c is not None:
        assert abs(k.c - paper_c) < 1e-15 * paper_c * 10
    val, _ = integrate.quad(lambda t: math.sin(t) ** 2 * float(k.g(t)), 0, math.pi,
                            limit=400, epsabs=1e-14, epsrel=1e-13)
    assert abs(math.pi / 2 * val - 1.0 / 6.0) < 1e-10
    assert abs(k.lam() - 1.0 / 6.0) < 1e-14


def test_family_matches_paper_b6_b7_pointwise():
    t = np.linspace(0.01, math.pi - 0.01, 50)
    b6 = 1.0 / (8 * math.pi * np.sin(t) * np.sin(t / 2))
    b7 = 1.0 / (6 * math.pi ** 2 * np.sin(t) * np.sin(t / 2) ** 2)
    b8 = 5 * np.cos(t / 2) / (192 * math.pi * np.sin(t) * np.sin(t / 2) ** 2.5)
    assert np.allclose(kernels.Kernel("family", 0.0).g(t), np.sin(t) * b6, rtol=1e-14)
    assert np.allclose(kernels.Kernel("family", 0.5).g(t), np.sin(t) * b7, rtol=1e-14)
    assert np.allclose(kernels.Kernel("b8").g(t), np.sin(t) * b8, rtol=1e-14)


@pytest.mark.parametrize("name,s", [("family", 0.0), ("family", 0.25), ("family", 0.5),
                                    ("family", 0.75), ("b5", 0.0), ("b8", 0.0)])
def test_taylor_moments_against_adaptive_quadrature(name, s):
    """Part I constants (Sec. 4.1) against an adaptive rule with the algebraic end weight."""
    k = kernels.Kernel(name, s)
    eps = math.pi / 1000
    A1, A2, A3 = k.taylor_moments(eps)
    alpha = {"family": -1.0 - 2 * s, "b5": 1.0, "b8": -2.5}[name]

    def q(fun, extra):
        # g(t) fun(t) = t^(alpha + extra) * smooth(t): integrate smooth against that weight
        def smooth(t):
            t = max(t, 1e-9)
            return float(k.g(t)) * fun(t) / t ** (alpha + extra)
        val, _ = integrate.quad(smooth, 0, eps, weight="alg", wvar=(alpha + extra, 0.0),
                                epsabs=0, epsrel=1e-13)
        return val

    r1 = q(lambda t: 2 * math.sin(t / 2) ** 2, 2.0)
    r2 = q(lambda t: 4 * math.sin(t / 2) ** 4, 4.0)
    r3 = q(lambda t: math.sin(t) ** 2, 2.0)
    for got, ref in [(A1, r1), (A2, r2), (A3, r3)]:
        assert abs(got - ref) <= 1e-10 * abs(ref)
