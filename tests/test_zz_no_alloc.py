"""bz_collide_noalloc: the collide for callers that cannot let the library allocate (GPU).

Its scratch lives in a fixed device array inside libbz instead of memory allocated by
the plan.  Checked through the C ABI against bz_collide (the allocating entry point) on
two calls in a row with different inputs, so contents left in the shared array by one call
must not leak into the next; the tolerance is the parity bar of the other GPU tests.
This file sorts last so that a run stopping at the first failure has run all the others.
"""
import numpy as np
import pytest

import bz_inputs as bi

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


@pytest.mark.parametrize("N,N_rho,M,dtype", [(16, 4, 12, torch.complex128),
                                             (32, 2, 32, torch.complex128),
                                             (24, 3, 12, torch.complex64)])
def test_noalloc_matches_collide_on_two_calls_in_a_row(bz, N, N_rho, M, dtype):
    L = 10.0
    plan = bz.bz_plan_create(N, L, bi.R_from_L(L), -1.0, 0.5, N_rho, M)
    fa = torch.from_numpy(bi.random_mixture(N, L, seed=101)).to("cuda", dtype)
    fb = torch.from_numpy(bi.two_maxwellians_c1(N, L)).to("cuda", dtype)
    ref_a, ref_b = torch.empty_like(fa), torch.empty_like(fb)
    bz.bz_collide(plan, fa, ref_a)
    bz.bz_collide(plan, fb, ref_b)
    q1, q2, q3 = torch.empty_like(fa), torch.empty_like(fa), torch.empty_like(fa)
    bz.bz_collide_noalloc(plan, fa, q1)
    bz.bz_collide_noalloc(plan, fb, q2)
    bz.bz_collide_noalloc(plan, fa, q3)
    torch.cuda.synchronize()
    ra, rb = ref_a.cpu().numpy(), ref_b.cpu().numpy()
    a1, a2, a3 = q1.cpu().numpy(), q2.cpu().numpy(), q3.cpu().numpy()
    assert _rel(a1, ra) <= TOL
    assert _rel(a2, rb) <= TOL
    assert np.array_equal(a3, a1)          # nothing of the previous call leaks through
    plan.close()


def test_noalloc_rejects_a_plan_larger_than_its_array(bz):
    N, L = 64, 10.0
    plan = bz.bz_plan_create(N, L, bi.R_from_L(L), 0.0, 0.5, 1, 12)
    f = torch.from_numpy(bi.random_mixture(N, L, seed=5)).cuda()
    q = torch.zeros_like(f)
    with pytest.raises(bz.BzError) as e:
        bz.bz_collide_noalloc(plan, f, q)
    assert e.value.code == 1              # BZ_ERR_ARG
    torch.cuda.synchronize()
    assert torch.count_nonzero(q).item() == 0
    plan.close()
