"""The 2D operator on the GPU (dim = 2: Sec. 4 with d = 2, Sec. 4.1 (i), kernels b1-b4 of
Sec. 5.2) against the 2D oracle.

Bars: the FP64 F table to 1e-10 of max|F|; the FP32 collide to relative L-infinity 1e-5 of
max|Q|; Table 1's N = 8 and N = 16 entries within the bands the oracle meets (the larger N
rows are below FP32 rounding of this pipeline).
"""
import math
import os

import numpy as np
import pytest

import bz_inputs as bi
from oracle import kernels, spectral2d as s2

pytestmark = pytest.mark.gpu
TOL = 1e-5
torch = pytest.importorskip("torch")
KIDS = {"b1": 3, "b2": 4, "b3": 5, "b4": 6}


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


def _plan(bz, N, L, R, gamma, name, N_rho, M):
    return bz.bz_plan_create_ex(N, L, R, gamma, 0.0, N_rho, M, kernel=KIDS[name], dim=2)


def _collide(bz, plan, fhat, p0=None, p1=None):
    f = torch.from_numpy(np.asarray(fhat)).to("cuda", dtype=torch.complex128)
    q = torch.empty_like(f)
    if p0 is None:
        bz.bz_collide(plan, f, q)
    else:
        bz.bz_collide_terms(plan, p0, p1, f, q)
    torch.cuda.synchronize()
    return q.cpu().numpy()


@pytest.mark.parametrize("name", list(KIDS))
def test_ftable2d_entries_match_oracle(bz, name):
    N, L = 16, 6.6
    R = 6.0
    plan = _plan(bz, N, L, R, 0.0, name, 4, 8)
    op = s2.OraclePlan2D(N, L, R, 0.0, kernels.Kernel2D(name), 4, 8)
    u = bi.SplitMix64(11).uniform(3 * 96)
    kidx = np.zeros((96, 3), dtype=np.int32)
    kidx[:, :2] = (u[:192].reshape(96, 2) * N).astype(np.int32)
    terms = (u[192:] * plan.P).astype(np.int32)
    got = bz.bz_ftable_entries(plan, torch.from_numpy(kidx).cuda(), torch.from_numpy(terms).cuda()).cpu().numpy()
    ref = op.F[terms, kidx[:, 0], kidx[:, 1]]
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(op.F))
    plan.close()


@pytest.mark.parametrize("N,name,gamma,N_rho,M", [(8, "b1", 0.0, 4, 8), (16, "b2", -1.0, 3, 12), (32, "b3", 0.0, 4, 16),
                                                  (64, "b4", -1.0, 2, 8), (32, "b4", 0.0, 32, 32)])
def test_collide2d_matches_oracle(bz, N, name, gamma, N_rho, M):
    L = 10.0
    R = bi.R_from_L(L)
    fhat = bi.random_mixture2d(N, L, seed=50 + N)
    plan = _plan(bz, N, L, R, gamma, name, N_rho, M)
    info = bz.bz_plan_pipeline(plan)
    assert info["pipeline"] == "fused" and info["clusters"] > 0
    got = _collide(bz, plan, fhat)
    ref = s2.collide2d(s2.OraclePlan2D(N, L, R, gamma, kernels.Kernel2D(name), N_rho, M), fhat)
    err = _rel(got, ref)
    print(f"2D N={N} {name} gamma={gamma} P={N_rho * M}: rel_Linf={err:.2e}")
    assert err <= TOL
    assert got[0, 0] == 0
    plan.close()


@pytest.mark.parametrize("N,name,lo,hi", [(8, "b1", 0.85, 1.05), (8, "b4", 0.8, 1.05), (16, "b1", 0.93, 1.03),
                                          (16, "b2", 1.0, 1.08)])
def test_table1_on_the_gpu(bz, N, name, lo, hi):
    R = 6.0
    L = bi.L_from_R(R)
    K = bi.bkw2d_K(0.0)
    ref = {l.split()[0]: l.split()[1:] for l in open(os.path.join(os.path.dirname(__file__), "golden",
                                                                   "table1_bkw2d.txt")) if l[0] != "#"}
    printed = float(ref[str(N)][list(KIDS).index(name)])
    plan = _plan(bz, N, L, R, 0.0, name, N, 32)
    Q = _collide(bz, plan, bi.bkw2d_fhat_samples(N, L, K))
    v = bi.grid2d_cells(N, L)
    V1, V2 = np.meshgrid(v, v, indexing="ij")
    err = float(np.max(np.abs(s2.eval2d(Q, L, v) - s2.bkw2d_Q(V1 ** 2 + V2 ** 2, K))))
    print(f"GPU Table 1 N={N} {name}: {err:.4e} (printed {printed:.4e}, ratio {err / printed:.3f})")
    assert lo <= err / printed <= hi
    plan.close()


def test_rk4_2d_term_ranges_and_refusals(bz):
    N = 32
    R = 6.0
    L = bi.L_from_R(R)
    f0 = bi.bkw2d_fhat(N, L, bi.bkw2d_K(1.0))
    plan = _plan(bz, N, L, R, 0.0, "b3", 4, 16)
    op = s2.OraclePlan2D(N, L, R, 0.0, kernels.Kernel2D("b3"), 4, 16)
    f = torch.from_numpy(f0.copy()).cuda()
    t = bz.bz_step_rk(plan, f, 1.0, 0.05, 2)
    torch.cuda.synchronize()
    assert abs(t - 1.1) < 1e-12
    ref = s2.rk4_2d(op, f0, 0.05, 2)
    err = _rel(f.cpu().numpy() - f0, ref - f0)
    print(f"2D RK4 2 steps: rel_Linf of the change = {err:.2e}")
    assert err <= TOL
    full = s2.collide2d(op, f0)
    parts = [_collide(bz, plan, f0, 0, 23), _collide(bz, plan, f0, 23, 64)]
    assert _rel(parts[0] + parts[1], full) <= 2 * TOL
    assert np.all(_collide(bz, plan, f0, 9, 9) == 0)
    fd = torch.from_numpy(f0).cuda()
    for call in (lambda: bz.bz_moments(plan, fd), lambda: bz.bz_batch_create(plan, 2, 0),
                 lambda: bz.bz_collide_noalloc(plan, fd, torch.empty_like(fd))):
        with pytest.raises(bz.BzError):
            call()
    plan.close()
    with pytest.raises(bz.BzError):                              # a 3D kernel id in 2D
        bz.bz_plan_create_ex(16, L, R, 0.0, 0.5, 2, 8, kernel=0, dim=2)
    with pytest.raises(bz.BzError):                              # a 2D kernel id in 3D
        bz.bz_plan_create_ex(16, L, R, 0.0, 0.5, 2, 12, kernel=3)
