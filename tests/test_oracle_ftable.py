"""Pins for the oracle's F(k, |q|, qhat) table (Sec. 4.1) -- CPU only."""
import math

import numpy as np
import pytest

import bz_inputs as bi
from oracle import ftable, kernels, quadrature

L = 10.0
R = bi.R_from_L(L)


def _sample_terms(n, seed):
    u = bi.SplitMix64(seed).uniform(3 * n)
    r = R * (0.05 + 0.95 * u[0::3])
    ct = 2 * u[1::3] - 1
    ph = 2 * math.pi * u[2::3]
    st = np.sqrt(1 - ct ** 2)
    q = np.stack([st * np.cos(ph), st * np.sin(ph), ct], 1)
    return r, q


def test_F_vanishes_at_k0_and_is_hermitian():
    """F(0, .) = 0 (Sec. 4, mass remark) and F(-k) = conj F(k) from eq. FF."""
    N = 8
    r, q = _sample_terms(3, 11)
    for kern in [kernels.Kernel("family", 0.5), kernels.Kernel("b8")]:
        F = ftable.ftable(N, L, r, q, kern)
        assert np.all(F[:, 0, 0, 0] == 0)
        ks = bi.signed_modes(N)
        inner = np.nonzero(ks != -N // 2)[0]
        neg = np.mod(-ks[inner], N)
        A = F[:, inner][:, :, inner][:, :, :, inner]
        B = F[:, neg][:, :, neg][:, :, :, neg]
        assert np.max(np.abs(A - np.conj(B))) < 1e-13


def test_F_cutoff_kernel_matches_closed_form():
    """b = 1/(4 pi): F = 4 pi C [exp(i a k.qhat) Sinc(a|k|) - 1] (eq. cutoff3D), Sinc(x) = sin x / x."""
    N = 16
    r, q = _sample_terms(4, 5)
    F = ftable.ftable(N, L, r, q, kernels.Kernel("b5"))
    ks = bi.signed_modes(N).astype(float)
    K1, K2, K3 = np.meshgrid(ks, ks, ks, indexing="ij")
    for p in range(len(r)):
        a = math.pi * r[p] / (2 * L)
        kq = K1 * q[p, 0] + K2 * q[p, 1] + K3 * q[p, 2]
        kn = np.sqrt(K1 ** 2 + K2 ** 2 + K3 ** 2)
        sinc = np.where(kn == 0, 1.0, np.sin(a * kn) / np.where(kn == 0, 1, a * kn))
        exact = np.exp(1j * a * kq) * sinc - 1.0
        assert np.max(np.abs(F[p] - exact)) < 1e-11


@pytest.mark.parametrize("name,s", [("family", 0.25), ("family", 0.5), ("family", 0.75), ("b8", 0.0)])
def test_F_matches_exact_funk_hecke_series_within_taylor_bound(name, s):
    """The split differs from the exact F only by the Taylor remainder on [0, eps]."""
    kern = kernels.Kernel(name, s)
    N = 16
    r, q = _sample_terms(3, 23)
    kk = np.array([[1, 0, 0], [3, -2, 5], [-8, -8, -8], [7, 7, -8], [0, -5, 2]])
    eig = ftable.funk_hecke_eigen(kern, 70)
    for p in range(len(r)):
        got = ftable.fentries(N, L, kk, np.full(len(kk), r[p]), np.tile(q[p], (len(kk), 1)), kern)
        for e, kv in enumerate(kk):
            z = math.pi * r[p] / (2 * L) * np.linalg.norm(kv)
            ex = ftable.f_exact_series(kv, r[p], q[p], L, kern, eig)
            bound = ftable.taylor_remainder_bound(z, kern) + 1e-11
            assert abs(got[e] - ex) <= bound, (kv, got[e], ex, bound)


def test_F_exact_phi_integral_matches_paper_midpoint_rule():
    """Part II with the exact phi integral (J0) equals the paper's phi midpoint rule."""
    kern = kernels.Kernel("family", 0.5)
    N = 16
    r, q = _sample_terms(2, 3)
    kk = np.array([[2, 1, -3], [-8, 7, 7], [5, -8, 0]])
    for p in range(2):
        got = ftable.fentries(N, L, kk, np.full(3, r[p]), np.tile(q[p], (3, 1)), kern)
        for e, kv in enumerate(kk):
            mid = ftable.f_phi_midpoint(kv, r[p], q[p], L, kern, nphi=96)
            assert abs(got[e] - mid) < 1e-11 * max(1.0, abs(mid))


def test_F_part2_rule_is_converged():
    kern = kernels.Kernel("family", 0.75)
    N = 16
    r, q = _sample_terms(2, 99)
    a = ftable.ftable(N, L, r, q, kern, npts=20)
    b = ftable.ftable(N, L, r, q, kern, npts=30)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


def test_F_entries_agree_with_table():
    kern = kernels.Kernel("family", 0.5)
    N = 8
    r, q = _sample_terms(2, 7)
    F = ftable.ftable(N, L, r, q, kern)
    ks = bi.signed_modes(N)
    idx = [(1, 2, 3), (7, 0, 4), (4, 4, 4)]
    for p in range(2):
        kk = np.array([[ks[i] for i in t] for t in idx])
        e = ftable.fentries(N, L, kk, np.full(3, r[p]), np.tile(q[p], (3, 1)), kern)
        for j, t in enumerate(idx):
            assert abs(e[j] - F[(p,) + t]) < 1e-15 * max(1, abs(e[j])) * 10
