"""Debye-Yukawa kernel and angular cutoffs on the GPU (Sec. 5.3-5.5) against the oracle, and
the paper's qualitative finding that the non-cutoff solutions lose their high-frequency
content faster than their cutoff versions (Figs. 3, 5 and the discontinuous-data figure).

Bars: F entries to 1e-10 of max|F|; collides to relative L-infinity 1e-5 of max|Q|.
"""
import math

import numpy as np
import pytest

import bz_inputs as bi
from oracle import ftable, kernels, spectral, spectral2d as s2

pytestmark = pytest.mark.gpu
TOL = 1e-5
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__._libbuild().build()
    import paper_2004_11239_gb300 as m
    return m


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _collide(bz, plan, fhat):
    f = torch.from_numpy(np.asarray(fhat)).to("cuda", dtype=torch.complex128)
    q = torch.empty_like(f)
    bz.bz_collide(plan, f, q)
    torch.cuda.synchronize()
    return q.cpu().numpy()


KID = {"family": 0, "b8": 2, "debye": 7}
CASES_3D = [("debye", 0.0, 0.0, 1.0), ("debye", 0.0, math.pi / 10, 1.0), ("family", 0.5, math.pi / 4, 0.0),
            ("b8", 0.0, math.pi / 10, 0.0)]


@pytest.mark.parametrize("name,s,theta0,gamma", CASES_3D)
def test_3d_ftable_entries_and_collide(bz, name, s, theta0, gamma):
    N, R = 16, 0.66
    L = bi.L_from_R(R)
    plan = bz.bz_plan_create_ex(N, L, R, gamma, s, 4, 12, kernel=KID[name], theta0=theta0)
    kern = kernels.Kernel(name, s, theta0=theta0)
    r, wr, q, wq, c = bz.bz_plan_terms(plan)
    u = bi.SplitMix64(7).uniform(4 * 64)
    kidx = (u[:192].reshape(64, 3) * N).astype(np.int32)
    terms = (u[192:] * plan.P).astype(np.int32)
    got = bz.bz_ftable_entries(plan, torch.from_numpy(kidx).cuda(), torch.from_numpy(terms).cuda()).cpu().numpy()
    ref = ftable.fentries(N, L, bi.signed_modes(N)[kidx], r[terms], q[terms], kern)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    fhat = bi.measure_valued_fhat(N, L, 3, rings=((0.2, 0.5),))
    Q = _collide(bz, plan, fhat)
    ref = spectral.collide(spectral.OraclePlan(N, L, R, gamma, kern, 4, 12), fhat)
    err = _rel(Q, ref)
    print(f"3D {name} s={s} theta0={theta0:.3f} gamma={gamma}: rel_Linf={err:.2e}")
    assert err <= TOL
    plan.close()


@pytest.mark.parametrize("theta0", [math.pi / 4, math.pi / 10])
def test_2d_cutoff_ftable_and_collide(bz, theta0):
    N, R = 32, 6.0
    L = bi.L_from_R(R)
    plan = bz.bz_plan_create_ex(N, L, R, 0.0, 0.0, 8, 16, kernel=bz.BZ_KERNEL_B3, dim=2, theta0=theta0)
    op = s2.OraclePlan2D(N, L, R, 0.0, kernels.Kernel2D("b3", theta0=theta0), 8, 16)
    u = bi.SplitMix64(9).uniform(3 * 64)
    kidx = np.zeros((64, 3), dtype=np.int32)
    kidx[:, :2] = (u[:128].reshape(64, 2) * N).astype(np.int32)
    terms = (u[128:] * plan.P).astype(np.int32)
    got = bz.bz_ftable_entries(plan, torch.from_numpy(kidx).cuda(), torch.from_numpy(terms).cuda()).cpu().numpy()
    assert np.max(np.abs(got - op.F[terms, kidx[:, 0], kidx[:, 1]])) <= 1e-10 * np.max(np.abs(op.F))
    fhat = bi.discontinuous2d_fhat(N, L)
    err = _rel(_collide(bz, plan, fhat), s2.collide2d(op, fhat))
    print(f"2D b3 theta0={theta0:.3f}: rel_Linf={err:.2e}")
    assert err <= TOL
    plan.close()


def _high(f, frac=0.25):
    """Energy of the modes with max |k_d| >= frac N (the discontinuity's and the deltas' tail)."""
    N = f.shape[0]
    k = np.abs(bi.signed_modes(N))
    kmax = np.maximum.reduce(np.meshgrid(*([k] * f.ndim), indexing="ij"))
    return float(np.sum(np.abs(f[kmax >= frac * N]) ** 2))


def _evolve(bz, plan, f0, dt, steps):
    f = torch.from_numpy(f0.copy()).cuda()
    bz.bz_step_rk(plan, f, 0.0, dt, steps)
    torch.cuda.synchronize()
    return f.cpu().numpy()


def test_non_cutoff_smooths_faster_2d_discontinuous(bz):
    """Sec. 5.5: b3 against b3 cut at theta0 = pi/4 and pi/10, discontinuous data, RK4 dt = 0.02."""
    N, R = 64, 6.0
    L = bi.L_from_R(R)
    f0 = bi.discontinuous2d_fhat(N, L)
    e = {}
    for label, theta0 in [("non-cutoff", 0.0), ("pi/10", math.pi / 10), ("pi/4", math.pi / 4)]:
        plan = bz.bz_plan_create_ex(N, L, R, 0.0, 0.0, 32, 32, kernel=bz.BZ_KERNEL_B3, dim=2, theta0=theta0)
        f = _evolve(bz, plan, f0, 0.02, 25)
        e[label] = _high(f)
        assert abs(f[0, 0] - f0[0, 0]) <= 1e-12 * abs(f0[0, 0])          # mass is kept
        plan.close()
    e0 = _high(f0)
    print(f"2D high-mode energy at t = 0.5 / t = 0: " + ", ".join(f"{k} {v / e0:.3f}" for k, v in e.items()))
    assert e["non-cutoff"] < e["pi/10"] < e["pi/4"] < e0


def test_non_cutoff_smooths_faster_3d_debye(bz):
    """Sec. 5.4: the Debye-Yukawa kernel against its cutoff (theta0 = pi/10), data of eq.
    initialdelta1, R = 0.66, gamma = 1, RK4 dt = 0.05."""
    N, R = 16, 0.66
    L = bi.L_from_R(R)
    f0 = bi.measure_valued_fhat(N, L, 3, rings=((0.2, 0.5),))
    e = {}
    for label, theta0 in [("non-cutoff", 0.0), ("cutoff", math.pi / 10)]:
        plan = bz.bz_plan_create_ex(N, L, R, 1.0, 0.0, 16, 12, kernel=bz.BZ_KERNEL_DEBYE, theta0=theta0)
        e[label] = _high(_evolve(bz, plan, f0, 0.05, 20))
        plan.close()
    e0 = _high(f0)
    print(f"3D Debye high-mode energy at t = 1 / t = 0: non-cutoff {e['non-cutoff'] / e0:.3f}, "
          f"cutoff {e['cutoff'] / e0:.3f}")
    assert e["non-cutoff"] < e["cutoff"]
