"""Term sharding on one GPU (GPU): the ranks' bz_collide_terms results over the host partition
add up to bz_collide (relative L-infinity 1e-6; only the FP32 rounding of how terms are grouped
into blocks differs), for the complex and real-data forms on the fused and chunked pipelines.
The all-reduce itself is covered on gloo ranks (test_shard.py)."""
import numpy as np
import pytest

import bz_inputs as bi

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


@pytest.mark.parametrize("N,N_rho,M,data", [(16, 4, 12, 0), (16, 4, 12, 1), (32, 4, 32, 1),
                                            (64, 2, 12, 0), (64, 2, 12, 1)])
def test_partition_sums_equal_the_whole_collide(bz, N, N_rho, M, data):
    L = 10.0
    plan = bz.bz_plan_create_ex(N, L, bi.R_from_L(L), -1.0, 0.5, N_rho, M, data=data)
    f = torch.from_numpy(bi.random_mixture(N, L, seed=31)).cuda()
    whole = torch.empty_like(f)
    bz.bz_collide(plan, f, whole)
    torch.cuda.synchronize()
    ref = whole.cpu().numpy()
    for world in (2, 3, 5):
        acc = np.zeros_like(ref)
        for rank in range(world):
            p0, p1 = bz.bz_partition_terms(plan.P, data, world, rank)
            q = torch.empty_like(f)
            bz.bz_collide_terms(plan, p0, p1, f, q)
            torch.cuda.synchronize()
            acc += q.cpu().numpy()
        err = float(np.max(np.abs(acc - ref)) / np.max(np.abs(ref)))
        print(f"N={N} P={plan.P} data={data} world={world}: rel_Linf={err:.2e}")
        assert err <= 1e-6
    plan.close()


def test_empty_range_gives_zero(bz):
    N, L = 16, 10.0
    plan = bz.bz_plan_create_ex(N, L, bi.R_from_L(L), 0.0, 0.5, 2, 12, data=1)
    f = torch.from_numpy(bi.random_mixture(N, L, seed=3)).cuda()
    q = torch.full_like(f, 1.0)
    bz.bz_collide_terms(plan, 8, 8, f, q)
    torch.cuda.synchronize()
    assert torch.count_nonzero(q).item() == 0
    plan.close()
