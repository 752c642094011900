"""Pins of the oracle's Debye-Yukawa kernel and angular cutoffs (Sec. 5.3-5.5; eqs.
ApproximatedDebye, ApproximatedDebyecutoff, b3cutoff), CPU only.

* Debye-Yukawa part I moments against a 30-digit mpmath quadrature.
* 3D F by the split against the Funk-Hecke series (no Taylor step): within the Taylor
  remainder bound for the Debye-Yukawa kernel, to rounding for cutoff kernels (whose part
  II starts at the cutoff; theta0 = pi/4 > 0.5 also exercises the equal-panel start).
* 2D F of b3 with cutoff against direct adaptive quadrature of eq. FF2D1.
* The discontinuous data of eq. disinitial has unit mass and zero momentum.
"""
import math

import numpy as np
import pytest

import bz_inputs as bi
from oracle import ftable, kernels

EPS = ftable.EPS_DEFAULT


def test_debye_part1_moments_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    A1, A2, A3 = kernels.Kernel("debye").taylor_moments(EPS)
    h = lambda t: mp.sin(t / 2)
    m1 = float(mp.quad(lambda t: h(t) * abs(mp.log(2 * h(t))), [0, EPS]))
    m2 = float(mp.quad(lambda t: 2 * h(t) ** 3 * abs(mp.log(2 * h(t))), [0, EPS]))
    m3 = float(mp.quad(lambda t: mp.sin(t) ** 2 * abs(mp.log(2 * h(t))) / (2 * h(t)), [0, EPS]))
    assert abs(A1 - m1) <= 1e-13 * m1 and abs(A2 - m2) <= 1e-13 * m2 and abs(A3 - m3) <= 1e-12 * m3


ENTRIES = (np.array([[1, 2, 0], [3, -1, 2], [-4, 4, 1], [0, 0, 5]], dtype=np.int32),
           np.array([0.5, 0.4, 0.6, 0.3]),
           np.array([[0, 0, 1.0], [0.6, 0.8, 0], [0.48, 0.6, 0.64], [0.0, 0.6, 0.8]]))


@pytest.mark.parametrize("kern", [kernels.Kernel("debye"), kernels.Kernel("debye", theta0=math.pi / 10),
                                  kernels.Kernel("family", 0.5, theta0=math.pi / 4),
                                  kernels.Kernel("b8", theta0=math.pi / 10)])
def test_3d_split_against_funk_hecke(kern):
    k, r, q = ENTRIES
    L = 0.73
    F = ftable.fentries(16, L, k, r, q, kern)
    for e in range(len(r)):
        ex = ftable.f_exact_series(k[e], r[e], q[e], L, kern)
        z = math.pi * r[e] / (2 * L) * float(np.linalg.norm(k[e]))
        bound = 0.0 if kern.theta0 > 0 else ftable.taylor_remainder_bound(z, kern)
        assert abs(F[e] - ex) <= bound + 1e-12 * max(1.0, abs(ex)), (kern, e, F[e], ex, bound)


@pytest.mark.parametrize("theta0", [math.pi / 4, math.pi / 10])
def test_2d_cutoff_against_direct_quadrature(theta0):
    from scipy.integrate import quad
    kern = kernels.Kernel2D("b3", theta0=theta0)
    N, L = 16, 6.6
    r = np.array([2.0, 5.0])
    q = np.array([[0.6, 0.8], [-1.0, 0.0]])
    F = ftable.ftable2d(N, L, r, q, kern)
    for p in range(2):
        a = math.pi * r[p] / (2 * L)
        for k1, k2 in [(1, 0), (3, -2), (-5, 7), (7, 7)]:
            x = a * (k1 * q[p, 0] + k2 * q[p, 1])
            y = a * (-k1 * q[p, 1] + k2 * q[p, 0])
            b = lambda t: float(kern.b(t))
            re = 2 * quad(lambda t: b(t) * (math.cos(x * (1 - math.cos(t))) * math.cos(y * math.sin(t)) - 1),
                          theta0, math.pi, epsabs=1e-14, epsrel=1e-13, limit=500)[0]
            im = 2 * quad(lambda t: b(t) * math.sin(x * (1 - math.cos(t))) * math.cos(y * math.sin(t)),
                          theta0, math.pi, epsabs=1e-14, epsrel=1e-13, limit=500)[0]
            got = F[p, k1 % N, k2 % N]
            assert abs(got - (re + 1j * im)) <= 1e-11 * max(1.0, abs(re + 1j * im))


def test_cutoff_kernels_have_no_taylor_part():
    assert kernels.Kernel("debye", theta0=0.3).taylor_moments(EPS) == (0.0, 0.0, 0.0)
    assert kernels.Kernel2D("b3", theta0=0.3).taylor_moments(EPS) == (0.0, 0.0, 0.0)


def test_discontinuous_data_moments():
    N, L = 64, 6.62
    f = bi.discontinuous2d_fhat(N, L)
    v = bi.grid(N, L)
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    fv = np.real(np.fft.ifftn(f * N * N * np.multiply.outer(*(np.where(bi.signed_modes(N) % 2 == 0, 1.0, -1.0),) * 2)))
    dv = (2 * L / N) ** 2
    assert abs(fv.sum() * dv - 1.0) < 1e-6                       # mass 1
    assert abs((fv * V2).sum() * dv) < 1e-6                      # no momentum across v_1 (grid ends at -L, not +L)
    assert abs(0.5 * (fv * (V1 ** 2 + V2 ** 2)).sum() * dv - 1.0) < 1e-3   # energy 1 (jump at v_1 = 0)
