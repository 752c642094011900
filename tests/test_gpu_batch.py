"""Batched instances (bz_batch_*) against the oracle and the single-instance path (GPU)."""
import numpy as np
import pytest

import bz_inputs as bi
from oracle import kernels, spectral

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


@pytest.mark.parametrize("N,N_rho,M,tb", [(16, 4, 12, 0), (32, 2, 12, 5), (24, 3, 12, 7)])
def test_batch_collide_matches_oracle_per_instance_and_is_batch_invariant(bz, N, N_rho, M, tb):
    L = 10.0
    R = bi.R_from_L(L)
    cap = 6
    gam = {4: 0.0, 1: -1.0, 3: -2.0, 0: 0.5}
    plan = bz.bz_plan_create(N, L, R, 0.0, 0.5, N_rho, M)
    batch = bz.bz_batch_create(plan, cap, tb)
    assert batch.terms_per_item >= 1
    for slot, g in gam.items():
        bz.bz_batch_set_gamma(batch, slot, g)
    f = np.zeros((cap, N, N, N), dtype=np.complex128)
    for slot in range(cap):
        f[slot] = bi.random_mixture(N, L, seed=100 + slot)
    fd = torch.from_numpy(f).cuda()
    qd = torch.zeros_like(fd)
    slots = [4, 1, 3, 0]
    bz.bz_batch_collide(batch, slots, fd, qd)
    torch.cuda.synchronize()
    q = qd.cpu().numpy()
    for slot in slots:
        op = spectral.OraclePlan(N, L, R, gam[slot], kernels.Kernel("family", 0.5), N_rho, M)
        ref = spectral.collide(op, f[slot])
        err = _rel(q[slot], ref)
        print(f"N={N} slot {slot} gamma={gam[slot]}: rel_Linf={err:.2e}")
        assert err <= TOL
    assert np.all(q[2] == 0) and np.all(q[5] == 0)        # inactive slots untouched
    # the same instance alone gives the same bits
    q_alone = torch.zeros_like(fd)
    bz.bz_batch_collide(batch, [3], fd, q_alone)
    torch.cuda.synchronize()
    assert np.array_equal(q_alone.cpu().numpy()[3], q[3])
    batch.close()
    plan.close()


def test_batch_rk4_matches_single_instance_rk4(bz):
    N = 16
    R = 6.0
    L = bi.L_from_R(R)
    plan = bz.bz_plan_create(N, L, R, 0.0, 0.5, 4, 12)
    batch = bz.bz_batch_create(plan, 3, 0)
    bz.bz_batch_set_gamma(batch, 2, -1.0)
    f = np.stack([bi.bkw_fhat(N, L, bi.bkw_K(6.5)), bi.random_mixture(N, L, seed=7, box=1.0),
                  bi.random_mixture(N, L, seed=8, box=1.0)])
    fd = torch.from_numpy(f).cuda()
    bz.bz_batch_step_rk(batch, [0, 2], fd, 0.05, 3)
    bz.bz_batch_step_rk(batch, [0, 2], fd, 0.05, 1)        # graph replay on a second call
    torch.cuda.synchronize()
    got = fd.cpu().numpy()
    assert np.array_equal(got[1], f[1])                    # inactive slot untouched
    for slot, g in [(0, 0.0), (2, -1.0)]:
        op = spectral.OraclePlan(N, L, R, g, kernels.Kernel("family", 0.5), 4, 12)
        ref = spectral.rk4(op, f[slot], 0.05, 4)
        err = _rel(got[slot] - f[slot], ref - f[slot])
        print(f"batch RK4 slot {slot}: rel_Linf of the change={err:.2e}")
        assert err <= TOL
        assert got[slot][0, 0, 0] == f[slot][0, 0, 0]     # mass mode exact
    batch.close()
    plan.close()


def test_batch_rejects_bad_slots(bz):
    plan = bz.bz_plan_create(16, 10.0, bi.R_from_L(10.0), 0.0, 0.5, 2, 12)
    batch = bz.bz_batch_create(plan, 4, 8)
    fd = torch.zeros((4, 16, 16, 16), dtype=torch.complex128, device="cuda")
    qd = torch.zeros_like(fd)
    for bad in ([4], [-1], [1, 1]):
        with pytest.raises(bz.BzError):
            bz.bz_batch_collide(batch, bad, fd, qd)
    batch.close()
    plan.close()


@pytest.mark.parametrize("N,N_rho,M,data", [(48, 2, 12, 0), (64, 1, 12, 1), (24, 3, 12, 1)])
def test_batches_of_chunked_plans(bz, N, N_rho, M, data):
    """A batch over a plan on the chunked pipeline (N = 24 real data, 48, 64): each slot with its
    own gamma (eq. approxG: c_p carries r^gamma) matches the oracle's operator of that gamma,
    a slot's result is the same bits alone and among others, and a batched RK4 step equals the
    plan's own RK4 on a plan built with that gamma within the FP32 bar."""
    L = 10.0
    R = bi.R_from_L(L)
    cap = 3
    gam = [0.0, -1.0, -2.0]
    plan = bz.bz_plan_create_ex(N, L, R, 0.0, 0.5, N_rho, M, data=data)
    assert bz.bz_plan_pipeline(plan)["pipeline"] == "chunked"
    batch = bz.bz_batch_create(plan, cap, 0)
    for slot, g in enumerate(gam):
        bz.bz_batch_set_gamma(batch, slot, g)
    f = np.stack([bi.random_mixture(N, L, seed=300 + slot) for slot in range(cap)])
    fd = torch.from_numpy(f).cuda()
    q = torch.empty_like(fd)
    bz.bz_batch_collide(batch, [0, 1, 2], fd, q)
    q1 = torch.zeros_like(fd)
    bz.bz_batch_collide(batch, [2], fd, q1)
    torch.cuda.synchronize()
    got = q.cpu().numpy()
    assert np.array_equal(q1.cpu().numpy()[2], got[2])           # alone = in the batch
    fn = spectral.collide_real if data else spectral.collide
    for slot in (1, 2):
        op = spectral.OraclePlan(N, L, R, gam[slot], kernels.Kernel("family", 0.5), N_rho, M)
        ref = fn(op, f[slot])
        err = _rel(got[slot], ref)
        print(f"chunked batch N={N} data={data} gamma={gam[slot]}: rel_Linf={err:.2e}")
        assert err <= TOL
    # RK4 through the batch against a plan with the slot's gamma
    g2 = bz.bz_plan_create_ex(N, L, R, -2.0, 0.5, N_rho, M, data=data)
    ref = fd[2].clone()
    bz.bz_step_rk(g2, ref, 0.0, 0.05, 2)
    cells = fd.clone()
    bz.bz_batch_step_rk(batch, [0, 2], cells, 0.05, 2)
    torch.cuda.synchronize()
    d = (cells[2] - fd[2]).cpu().numpy()
    dr = (ref - fd[2]).cpu().numpy()
    assert _rel(d, dr) <= TOL
    assert torch.equal(cells[1], fd[1])                           # inactive slot untouched
    g2.close()
    batch.close()
    plan.close()
