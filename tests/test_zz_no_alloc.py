"""bz_collide_noalloc: the collide for callers that cannot let the library allocate (GPU).

Its scratch lives in a fixed device array inside libbz instead of memory allocated by
the plan.  Checked through the C ABI against bz_collide (the allocating entry point) on
two calls in a row with different inputs, so contents left in the shared array by one call
must not leak into the next; the tolerance is the parity bar of the other GPU tests.
This file sorts last so that a run stopping at the first failure has run all the others.
"""
import math

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


SCRATCH = 8 << 20          # BZ_NOALLOC_SCRATCH_BYTES


def _terms_per_chunk(N, h64):
    """Terms per chunk as the header states the array's layout: 8 N^3 bytes each for the FP32
    input and h, 16 N^3 for the FP64 accumulator, 16 N^3 more where h is formed in FP64."""
    field = 8 * N ** 3
    fixed = 4 * field + (2 * field if h64 else 0)
    return (SCRATCH - fixed) // field


@pytest.mark.parametrize("N,N_rho,M,dtype", [(16, 4, 12, torch.complex128),
                                             (32, 2, 32, torch.complex128),
                                             (24, 3, 12, torch.complex64),
                                             (48, 2, 12, torch.complex64),
                                             (8, 4, 12, torch.complex128)])
def test_noalloc_matches_collide_on_two_calls_in_a_row(bz, N, N_rho, M, dtype):
    L = 10.0
    plan = bz.bz_plan_create(N, L, bi.R_from_L(L), -1.0, 0.5, N_rho, M)
    if N == 48:
        # the chunked pipeline with FP32 h: five terms per chunk, so the 24 terms take five chunks
        assert bz.bz_plan_pipeline(plan)["pipeline"] == "chunked"
        T = _terms_per_chunk(N, False)
        assert T == 5 and math.ceil(plan.P / T) > 1
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


def test_noalloc_matches_the_oracle_on_an_under_resolved_mixture(bz):
    """The same operator as bz_collide (h formed in FP64 on the fused pipeline): within the FP32
    bar of the FP64 oracle on the N = 32 mixture where FP32-formed h alone exceeds it."""
    N, L = 32, 10.0
    R = bi.R_from_L(L)
    fhat = bi.random_mixture(N, L, seed=63)
    plan = bz.bz_plan_create(N, L, R, -1.0, 0.5, 2, 12)
    f = torch.from_numpy(fhat).cuda()
    q = torch.empty_like(f)
    bz.bz_collide_noalloc(plan, f, q)
    bz.bz_collide_noalloc(plan, f, q)
    torch.cuda.synchronize()
    ref = spectral.collide(spectral.OraclePlan(N, L, R, -1.0, kernels.Kernel("family", 0.5), 2, 12), fhat)
    err = _rel(q.cpu().numpy(), ref)
    print(f"noalloc N=32 under-resolved mixture: rel_Linf={err:.2e}")
    assert err <= TOL
    plan.close()


def test_noalloc_refuses_split_bf16_plans(bz):
    """A split-BF16 plan is served by bz_collide only: BZ_ERR_UNSUPPORTED, Qhat untouched."""
    N, L = 32, 10.0
    plan = bz.bz_plan_create_ex(N, L, bi.R_from_L(L), 0.0, 0.5, 2, 12, precision=bz.BZ_PREC_BF16X3)
    f = torch.from_numpy(bi.random_mixture(N, L, seed=5)).cuda()
    q = torch.zeros_like(f)
    with pytest.raises(bz.BzError) as e:
        bz.bz_collide_noalloc(plan, f, q)
    assert e.value.code == 7              # BZ_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.count_nonzero(q).item() == 0
    plan.close()
