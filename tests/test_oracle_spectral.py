"""Pins for the oracle's spectral operator (Sec. 2, Sec. 4, Sec. 5.1) -- CPU only."""
import math
import os

import numpy as np
import pytest

import bz_inputs as bi
from oracle import kernels, spectral

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_bkw3d.txt")


def test_dft3_is_the_library_dft():
    """The written-out DFT equals the library FFT (numpy) in both directions."""
    for N in (6, 8, 12):
        x = bi.random_fhat(N, seed=N)
        assert np.allclose(spectral.dft3(x, -1), np.fft.fftn(x), atol=1e-12)
        assert np.allclose(spectral.dft3(x, +1), np.fft.ifftn(x) * N ** 3, atol=1e-12)


@pytest.fixture(scope="module")
def plan8():
    L = 6.0
    return spectral.OraclePlan(8, L, bi.R_from_L(L), -1.0, kernels.Kernel("family", 0.5), 3, 12)


@pytest.mark.parametrize("padded", [False, True])
def test_fft_form_equals_direct_weighted_sum(plan8, padded):
    """Eq. realQ evaluated with DFTs equals the double sum of eq. sum with G from eq. approxG."""
    f = bi.random_fhat(8, seed=4)
    Q = spectral.collide(plan8, f, padded=padded)
    Qd = spectral.direct_sum(plan8, f, padded=padded)
    assert np.max(np.abs(Q - Qd)) < 1e-12 * np.max(np.abs(Qd))


def test_mass_mode_is_exactly_zero(plan8):
    """Sec. 4 remark: F(0, ., .) = 0 hence Qhat_0 = 0 exactly."""
    for seed in range(3):
        Q = spectral.collide(plan8, bi.random_mixture(8, plan8.L, seed, box=1.0))
        assert Q[0, 0, 0] == 0


@pytest.fixture(scope="module")
def plan16():
    L = 10.0
    return spectral.OraclePlan(16, L, bi.R_from_L(L), 0.0, kernels.Kernel("family", 0.5), 16, 12)


def test_conservation_and_symmetry_n16(plan16):
    """Q conserves momentum and energy to quadrature accuracy (Sec. 1) and is Hermitian for real f."""
    L = plan16.L
    f = bi.random_mixture(16, L, seed=7, box=1.5)
    f[8, :, :] = 0          # no Nyquist content: the non-Nyquist modes are closed under k -> -k
    f[:, 8, :] = 0
    f[:, :, 8] = 0
    Q = spectral.collide(plan16, f)
    mQ = spectral.moments(Q, L)
    # scale: the positive part of |v|^2 Q
    v2 = spectral.grid_v2(16, L)
    Qv = spectral.to_grid(Q, L).real
    scale = np.sum(np.abs(Qv) * v2) * (2 * L / 16) ** 3
    assert abs(mQ[0]) < 1e-14
    assert np.max(np.abs(mQ[1:4])) < 2e-3 * scale
    assert abs(mQ[4]) < 2e-3 * scale
    ks = bi.signed_modes(16)
    inner = np.nonzero(ks != -8)[0]
    neg = np.mod(-ks[inner], 16)
    A = Q[np.ix_(inner, inner, inner)]
    B = Q[np.ix_(neg, neg, neg)]
    assert np.max(np.abs(A - np.conj(B))) < 1e-12 * np.max(np.abs(Q))


def test_maxwellian_is_near_equilibrium():
    """Q(M, M) = 0 for a Maxwellian (Sec. 1): the residual shrinks as the sphere rule refines and
    ends far below Q of a non-equilibrium mixture."""
    R = 6.0
    L = bi.L_from_R(R)
    M = bi.gaussian_mixture_fhat(16, L, [1.0], [(0.0, 0.0, 0.0)], [1.0])
    f = bi.gaussian_mixture_fhat(16, L, [0.5, 0.5], [(1.0, 0, 0), (-1.0, 0, 0)], [0.7, 0.7])
    res = []
    for Mq in (12, 72):
        plan = spectral.OraclePlan(16, L, R, 0.0, kernels.Kernel("family", 0.5), 16, Mq)
        res.append(np.max(np.abs(spectral.collide(plan, M))))
    qf = np.max(np.abs(spectral.collide(plan, f)))
    assert res[1] < 0.1 * res[0]
    assert res[1] < 1e-2 * qf


def test_bkw_closed_forms_are_consistent():
    """Eq. QQ equals the time derivative of eq. BKW with K' = lambda (1 - K) (eq. odeK)."""
    v2 = np.linspace(0, 30, 200)
    lam = 1.0 / 6.0
    for t in (5.6, 6.5, 9.0):
        h = 1e-4
        Kp, Km = bi.bkw_K(t + h), bi.bkw_K(t - h)
        fd = (spectral.bkw_f(v2, Kp) - spectral.bkw_f(v2, Km)) / (2 * h)
        ex = spectral.bkw_Q(v2, bi.bkw_K(t), lam)
        assert np.max(np.abs(fd - ex)) < 1e-8 * np.max(np.abs(ex)) + 1e-12


def test_moments_of_gaussians():
    """Mass, momentum and energy of a Gaussian: m, m u, m (|u|^2 + 3 T)."""
    L, N = 10.0, 48
    u, T, m = (0.7, -0.4, 1.1), 0.8, 1.3
    f = bi.gaussian_mixture_fhat(N, L, [m], [u], [T])
    mo = spectral.moments(f, L)
    ref = [m, m * u[0], m * u[1], m * u[2], m * (sum(x * x for x in u) + 3 * T)]
    assert np.allclose(mo, ref, rtol=1e-9, atol=1e-10)


def _bkw_error(N, N_rho, M, kern):
    R = 6.0
    L = bi.L_from_R(R)
    K = bi.bkw_K(6.5)
    plan = spectral.OraclePlan(N, L, R, 0.0, kern, N_rho, M)
    Q = spectral.collide(plan, bi.bkw_fhat(N, L, K))
    Qv = spectral.to_grid(Q, L)
    return np.max(np.abs(Qv - spectral.bkw_Q(spectral.grid_v2(N, L), K)))


@pytest.mark.parametrize("name,s", [("b5", 0), ("family", 0.0), ("family", 0.5), ("b8", 0)])
def test_bkw_error_small_at_n16(name, s):
    err = _bkw_error(16, 16, 12, kernels.Kernel(name, s))
    assert err < 3e-3          # |Q_ext| ~ 2e-2


@pytest.mark.slow
@pytest.mark.parametrize("col,name,s", [(3, "family", 0.5), (4, "b8", 0)])
def test_bkw_error_reproduces_paper_table2(col, name, s):
    """Sec. 5.3 Table 2, N_qhat = 12 row: the 12-point rule here is the icosahedron."""
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    paper = float(next(r for r in rows if r[0] == "12")[col])
    err = _bkw_error(32, 32, 12, kernels.Kernel(name, s))
    assert 0.7 * paper < err < 1.4 * paper, (err, paper)


def test_rk4_is_fourth_order():
    """Classical RK4 (Sec. 5.2): halving dt divides the error by about 16."""
    L = 6.0
    plan = spectral.OraclePlan(8, L, bi.R_from_L(L), 0.0, kernels.Kernel("family", 0.5), 3, 12)
    f0 = bi.random_mixture(8, L, seed=1, box=1.0)
    Tend = 1.0
    ref = spectral.rk4(plan, f0, Tend / 256, 256)
    e = [np.max(np.abs(spectral.rk4(plan, f0, Tend / n, n) - ref)) for n in (8, 16, 32)]
    assert 14 < e[0] / e[1] < 20 and 14 < e[1] / e[2] < 20


def test_rk4_steps_one_step_is_the_fourth_order_taylor_polynomial():
    """One classical RK4 step (Sec. 5.2) on the linear system y' = A y multiplies y by
    1 + Z + Z^2/2 + Z^3/6 + Z^4/24 exactly (Z = dt A): a wrong stage weight or a stage taken at
    the wrong point changes a coefficient of this polynomial."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    y0 = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    dt = 0.3
    Z = dt * A
    I = np.eye(4)
    poly = I + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    got = spectral.rk4_steps(lambda y: A @ y, y0, dt, 1)
    assert np.allclose(got, poly @ y0, rtol=0, atol=1e-13 * np.abs(poly @ y0).max())
    # nsteps steps apply the polynomial nsteps times
    got3 = spectral.rk4_steps(lambda y: A @ y, y0, dt, 3)
    assert np.allclose(got3, poly @ poly @ poly @ y0, rtol=0, atol=1e-12 * np.abs(got3).max())


def test_rk4_real_is_fourth_order():
    """The real-data RK4 (Sec. 5.2 on the real-data reading, `rk4_real`): halving dt divides
    the error by about 16."""
    L = 6.0
    plan = spectral.OraclePlan(8, L, bi.R_from_L(L), 0.0, kernels.Kernel("family", 0.5), 3, 12)
    f0 = bi.random_mixture(8, L, seed=1, box=1.0)
    Tend = 1.0
    ref = spectral.rk4_real(plan, f0, Tend / 256, 256)
    e = [np.max(np.abs(spectral.rk4_real(plan, f0, Tend / n, n) - ref)) for n in (8, 16, 32)]
    assert 14 < e[0] / e[1] < 20 and 14 < e[1] / e[2] < 20, e


def test_collide_at_equals_collide_at_those_modes():
    """`collide_at` (all terms, a few output modes, F supplied per mode) equals `collide` at the
    same modes, for the complex operator and the real-data band; the modes include both ends of
    every axis."""
    from oracle import ftable
    L = 6.0
    N = 8
    plan = spectral.OraclePlan(N, L, bi.R_from_L(L), -1.0, kernels.Kernel("family", 0.5), 3, 12)
    f = bi.random_mixture(N, L, seed=9, box=1.5)
    u = bi.SplitMix64(4).uniform(3 * 20)
    kidx = np.concatenate([np.array([[0, 0, 0], [N - 1, N // 2, 1], [N // 2, N - 1, N // 2]]),
                           (u.reshape(20, 3) * N).astype(int)])
    ks = spectral.signed(N)[kidx]
    P = plan.P
    F_at = ftable.fentries(N, L, np.repeat(ks, P, axis=0), np.tile(plan.r, len(ks)),
                           np.tile(plan.q, (len(ks), 1)), plan.kernel).reshape(len(ks), P)
    for g in (f, spectral.real_band(f)):
        full = spectral.collide(plan, g)
        got = spectral.collide_at(plan, g, kidx, F_at)
        want = full[kidx[:, 0], kidx[:, 1], kidx[:, 2]]
        assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(full))
    # a term range with the matching columns of F
    part = spectral.collide(plan, f, 5, 17)
    got = spectral.collide_at(plan, f, kidx, F_at[:, 5:17], 5, 17)
    assert np.max(np.abs(got - part[kidx[:, 0], kidx[:, 1], kidx[:, 2]])) < 1e-12 * np.max(np.abs(part))
