"""Split-BF16 tensor-core form (BZ_PREC_BF16X3) against the FP64 oracle (GPU).

Bar: relative L-infinity error max|Q_gpu - Q_oracle| / max|Q_oracle| <= 1e-3, the accuracy
target of the split-BF16 form; every run also checks that no bounded device wait gave up.
The per-axis DFTs keep about 16 significant bits (x_hi w_hi + x_lo w_hi + x_hi w_lo), so
the expected error is a few 1e-4 where the FP32 form reaches a few 1e-6.
"""
import numpy as np
import pytest

import bz_inputs as bi
from oracle import kernels, spectral

pytestmark = pytest.mark.gpu
TOL = 1e-3
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


def _mixed_plan(bz, N, L, R, gamma, s, N_rho, M, kernel=0):
    return bz.bz_plan_create_ex(N, L, R, gamma, s, N_rho, M, kernel=kernel, precision=bz.BZ_PREC_BF16X3)


def _collide(bz, plan, fhat, p0=None, p1=None):
    f = torch.from_numpy(np.asarray(fhat)).to("cuda", dtype=torch.complex128)
    q = torch.empty_like(f)
    if p0 is None:
        bz.bz_collide(plan, f, q)
    else:
        bz.bz_collide_terms(plan, p0, p1, f, q)
    torch.cuda.synchronize()
    return q.cpu().numpy()


CASES = [
    # gamma, s, kernel name, kernel id, N_rho, M, data
    (-1.0, 0.5, "family", 0, 2, 12, "mixture"),
    (0.0, 0.5, "family", 0, 3, 12, "two_maxwellians"),
    (0.0, 0.25, "family", 0, 2, 32, "bkw"),
    (-2.0, 0.0, "b8", 2, 2, 12, "mixture"),
]


@pytest.mark.parametrize("gamma,s,name,kid,N_rho,M,data", CASES)
def test_bf16x3_collide_matches_oracle(bz, gamma, s, name, kid, N_rho, M, data):
    N = 32
    if data == "bkw":
        R = 6.0
        L = bi.L_from_R(R)
        fhat = bi.bkw_fhat(N, L, bi.bkw_K(6.5))
    else:
        L = 10.0
        R = bi.R_from_L(L)
        fhat = bi.random_mixture(N, L, seed=63) if data == "mixture" else bi.two_maxwellians_c1(N, L)
    plan = _mixed_plan(bz, N, L, R, gamma, s, N_rho, M, kid)
    info = bz.bz_plan_pipeline(plan)
    assert info["pipeline"] == "fused" and info["cluster"] == 8
    got = _collide(bz, plan, fhat)
    assert bz.bz_plan_device_errors(plan) == 0
    ref = spectral.collide(spectral.OraclePlan(N, L, R, gamma, kernels.Kernel(name, s), N_rho, M), fhat)
    err = _rel(got, ref)
    print(f"BF16X3 N=32 {data} gamma={gamma} {name} s={s} P={N_rho * M}: rel_Linf={err:.2e}")
    assert err <= TOL
    assert got[0, 0, 0] == 0                  # alpha_p(0) = 0 for every term: mass is conserved
    plan.close()


def test_bf16x3_term_ranges_and_empty_range(bz):
    N, L = 32, 10.0
    R = bi.R_from_L(L)
    fhat = bi.random_mixture(N, L, seed=21)
    plan = _mixed_plan(bz, N, L, R, 0.0, 0.5, 2, 12)
    op = spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 2, 12)
    full = spectral.collide(op, fhat)
    scale = np.max(np.abs(full))
    parts = []
    for p0, p1 in [(0, 7), (7, 24)]:
        got = _collide(bz, plan, fhat, p0, p1)
        ref = spectral.collide(op, fhat, p0, p1)
        err = float(np.max(np.abs(got - ref)) / scale)
        print(f"BF16X3 terms [{p0},{p1}): error / max|Q| = {err:.2e}")
        assert err <= TOL
        parts.append(got)
    assert float(np.max(np.abs(parts[0] + parts[1] - full)) / scale) <= 2 * TOL
    empty = _collide(bz, plan, fhat, 5, 5)
    assert np.all(empty == 0)
    assert bz.bz_plan_device_errors(plan) == 0
    plan.close()


def test_bf16x3_rk4_matches_oracle_trajectory(bz):
    N = 32
    R = 6.0
    L = bi.L_from_R(R)
    f0 = bi.bkw_fhat(N, L, bi.bkw_K(6.5))
    plan = _mixed_plan(bz, N, L, R, 0.0, 0.5, 2, 12)
    f = torch.from_numpy(f0.copy()).cuda()
    t = bz.bz_step_rk(plan, f, 6.5, 0.05, 2)
    torch.cuda.synchronize()
    assert abs(t - 6.6) < 1e-12
    got = f.cpu().numpy()
    op = spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 2, 12)
    ref = spectral.rk4(op, f0, 0.05, 2)
    err = _rel(got - f0, ref - f0)
    print(f"BF16X3 RK4 2 steps: rel_Linf of the change = {err:.2e}")
    assert err <= TOL
    assert bz.bz_plan_device_errors(plan) == 0
    plan.close()


def test_bf16x3_batch_matches_oracle_and_is_batch_invariant(bz):
    N, L = 32, 10.0
    R = bi.R_from_L(L)
    plan = _mixed_plan(bz, N, L, R, 0.0, 0.5, 2, 12)
    cap = 4
    batch = bz.bz_batch_create(plan, cap, 5)
    gam = {2: -1.0, 0: 0.0, 3: -2.0}
    for slot, g in gam.items():
        bz.bz_batch_set_gamma(batch, slot, g)
    f = np.stack([bi.random_mixture(N, L, seed=300 + b) for b in range(cap)])
    fd = torch.from_numpy(f).cuda()
    qd = torch.zeros_like(fd)
    bz.bz_batch_collide(batch, [2, 0, 3], fd, qd)
    torch.cuda.synchronize()
    q = qd.cpu().numpy()
    for slot, g in gam.items():
        ref = spectral.collide(spectral.OraclePlan(N, L, R, g, kernels.Kernel("family", 0.5), 2, 12), f[slot])
        err = _rel(q[slot], ref)
        print(f"BF16X3 batch slot {slot} gamma={g}: rel_Linf={err:.2e}")
        assert err <= TOL
    assert np.all(q[1] == 0)
    alone = torch.zeros_like(fd)
    bz.bz_batch_collide(batch, [3], fd, alone)
    torch.cuda.synchronize()
    assert np.array_equal(alone.cpu().numpy()[3], q[3])      # the same bits alone and in the batch
    assert bz.bz_plan_device_errors(plan) == 0
    batch.close()
    plan.close()


def test_bf16x3_and_fp32_forms_agree_at_full_size(bz):
    """The bench's workload (N = 32, P = 1024, BKW at t = 6.5): the split-BF16 form against the
    FP32 form (itself held to 1e-5 of the oracle at this size) and the exact mass mode."""
    N, R = 32, 6.0
    L = bi.L_from_R(R)
    fhat = bi.bkw_fhat(N, L, bi.bkw_K(6.5))
    pm = _mixed_plan(bz, N, L, R, 0.0, 0.5, 32, 32)
    pf = bz.bz_plan_create(N, L, R, 0.0, 0.5, 32, 32)
    gm = _collide(bz, pm, fhat)
    gf = _collide(bz, pf, fhat)
    err = _rel(gm, gf)
    print(f"BF16X3 vs FP32, N=32 P=1024 BKW: rel_Linf={err:.2e}")
    assert err <= TOL - 1e-5
    assert gm[0, 0, 0] == 0
    assert bz.bz_plan_device_errors(pm) == 0
    pm.close()
    pf.close()
