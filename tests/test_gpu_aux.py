"""Failure detection and checkpoint/resume on the GPU, without a fault (GPU).

* Non-finite results: a host-made NaN in fhat reaches Qhat; the plan's flag reports it once
  (bz_plan_check_finite) and is cleared; bz_moments returns BZ_ERR_NONFINITE; RK steps and batch
  calls raise the same flag; finite inputs never do.
* Bounded waits: bz_plan_wait_selftest makes one wait on a barrier that nothing completes run
  out; bz_plan_device_errors then reports it and the context stays usable (a collide after it
  still matches the oracle).
* Checkpoint/resume (RK4, Sec. 5.2): six steps in one call equal three steps, a checkpoint, a
  plan rebuilt from the file and three more steps, bit for bit (complex128 state).
"""
import os
import tempfile

import numpy as np
import pytest

import bz_inputs as bi
from oracle import kernels, spectral

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__._libbuild().build()
    import paper_2004_11239_gb300 as m
    return m


@pytest.mark.parametrize("N,data", [(16, 0), (16, 1), (64, 1)])
def test_nan_input_raises_the_nonfinite_flag_once(bz, N, data):
    L = 10.0
    plan = bz.bz_plan_create_ex(N, L, bi.R_from_L(L), 0.0, 0.5, 2, 12, data=data)
    f = torch.from_numpy(bi.random_mixture(N, L, seed=4)).cuda()
    q = torch.empty_like(f)
    bz.bz_collide(plan, f, q)
    assert bz.bz_plan_check_finite(plan) == 0
    g = f.clone()
    g[0, 0, 3] = complex(float("nan"), 0.0)         # on an axis line: the moments see it too
    bz.bz_collide(plan, g, q)
    assert bz.bz_plan_check_finite(plan) == 1
    assert bz.bz_plan_check_finite(plan) == 0            # cleared by the check
    with pytest.raises(bz.BzError) as e:
        bz.bz_moments(plan, g)
    assert e.value.code == 5                              # BZ_ERR_NONFINITE
    assert all(np.isfinite(bz.bz_moments(plan, f)))
    if N == 16:
        h = g.clone()
        bz.bz_step_rk(plan, h, 0.0, 0.01, 1)
        assert bz.bz_plan_check_finite(plan) == 1
        batch = bz.bz_batch_create(plan, 2, 0)
        cells = torch.stack([f, g])
        out = torch.empty_like(cells)
        bz.bz_batch_collide(batch, [0], cells, out)
        assert bz.bz_plan_check_finite(plan) == 0        # slot 1 (NaN) not active
        bz.bz_batch_collide(batch, [0, 1], cells, out)
        assert bz.bz_plan_check_finite(plan) == 1
        batch.close()
    plan.close()


def test_bounded_wait_runs_out_and_the_context_stays_usable(bz):
    N, L = 16, 10.0
    R = bi.R_from_L(L)
    plan = bz.bz_plan_create(N, L, R, 0.0, 0.5, 2, 12)
    assert bz.bz_plan_device_errors(plan) == 0
    bz.bz_plan_wait_selftest(plan, 20000)
    torch.cuda.synchronize()
    assert bz.bz_plan_device_errors(plan) == 1
    fhat = bi.two_maxwellians_c1(N, L)
    f = torch.from_numpy(fhat).cuda()
    q = torch.empty_like(f)
    bz.bz_collide(plan, f, q)
    torch.cuda.synchronize()
    ref = spectral.collide(spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 2, 12), fhat)
    assert np.max(np.abs(q.cpu().numpy() - ref)) / np.max(np.abs(ref)) <= 1e-5
    with pytest.raises(bz.BzError):
        bz.bz_plan_wait_selftest(plan, 0)
    plan.close()


@pytest.mark.parametrize("N,data", [(16, 0), (32, 1), (48, 1)])
def test_checkpoint_resume_is_bitwise_identical(bz, N, data):
    L = 10.0
    R = bi.R_from_L(L)
    plan = bz.bz_plan_create_ex(N, L, R, -1.0, 0.5, 2, 12, data=data)
    f0 = torch.from_numpy(bi.random_mixture(N, L, seed=77)).cuda()
    whole = f0.clone()
    bz.bz_step_rk(plan, whole, 0.0, 0.02, 6)
    part = f0.clone()
    t = bz.bz_step_rk(plan, part, 0.0, 0.02, 3)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "state.bzck")
        bz.bz_checkpoint_write(plan, part, t, path)
        plan.close()                                     # the solve resumes in a new plan
        desc, t_file = bz.bz_checkpoint_plan_desc(path)
        assert t_file == t and desc.N == N and desc.data == data
        plan2 = bz.bz_plan_create_from_desc(desc)
        resumed = torch.zeros_like(f0)
        t2 = bz.bz_checkpoint_read(plan2, path, resumed)
        assert t2 == t
        bz.bz_step_rk(plan2, resumed, t2, 0.02, 3)
        torch.cuda.synchronize()
        assert torch.equal(resumed, whole)
        # a plan of another operator refuses the file
        other = bz.bz_plan_create_ex(N, L, R, 0.0, 0.5, 2, 12, data=data)
        with pytest.raises(bz.BzError) as e:
            bz.bz_checkpoint_read(other, path, resumed)
        assert e.value.code == 1
        other.close()
        plan2.close()
