"""Galerkin-exact (padded, l + m = k without wrap-around) form on the GPU (BZ_CONV_PADDED)
against the oracle's padded form, whose definition the direct O(N^6) sum pins at N = 8.

Bar: relative L-infinity 1e-5 of max|Q| (the FP32 pipeline on the 2N grid).  The padded
plan runs the fused kernel for 2N <= 32 and the chunked pipeline for 2N = 48, 64.
"""
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


def _padded_plan(bz, N, L, R, gamma, s, N_rho, M):
    return bz.bz_plan_create_ex(N, L, R, gamma, s, N_rho, M, conv=bz.BZ_CONV_PADDED)


def _collide(bz, plan, fhat, p0=None, p1=None, dtype=torch.complex128):
    f = torch.from_numpy(np.asarray(fhat)).to("cuda", dtype=dtype)
    q = torch.empty_like(f)
    if p0 is None:
        bz.bz_collide(plan, f, q)
    else:
        bz.bz_collide_terms(plan, p0, p1, f, q)
    torch.cuda.synchronize()
    return q.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("N,N_rho,M,gamma,pipe", [(8, 3, 12, 0.0, "fused"), (16, 2, 12, -1.0, "fused"),
                                                  (24, 1, 12, 0.0, "chunked"), (32, 1, 12, -2.0, "chunked")])
def test_padded_collide_matches_oracle(bz, N, N_rho, M, gamma, pipe):
    L = 10.0
    R = bi.R_from_L(L)
    fhat = bi.random_mixture(N, L, seed=70 + N, box=2.0)
    plan = _padded_plan(bz, N, L, R, gamma, 0.5, N_rho, M)
    assert bz.bz_plan_pipeline(plan)["pipeline"] == pipe
    got = _collide(bz, plan, fhat)
    op = spectral.OraclePlan(N, L, R, gamma, kernels.Kernel("family", 0.5), N_rho, M)
    ref = spectral.collide(op, fhat, padded=True)
    err = _rel(got, ref)
    circ = spectral.collide(op, fhat)
    print(f"padded N={N} ({pipe} at {2 * N}) P={N_rho * M}: rel_Linf={err:.2e}; "
          f"padded vs circular differ by {_rel(ref, circ):.2e}")
    assert err <= TOL
    assert got[0, 0, 0] == 0
    plan.close()


def test_padded_term_ranges_c64_and_moments(bz):
    N, L = 16, 10.0
    R = bi.R_from_L(L)
    fhat = bi.random_mixture(N, L, seed=5)
    plan = _padded_plan(bz, N, L, R, 0.0, 0.25, 2, 12)
    op = spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.25), 2, 12)
    full = spectral.collide(op, fhat, padded=True)
    scale = np.max(np.abs(full))
    for p0, p1 in [(0, 5), (5, 24), (9, 9)]:
        got = _collide(bz, plan, fhat, p0, p1)
        ref = spectral.collide(op, fhat, p0, p1, padded=True)
        assert float(np.max(np.abs(got - ref)) / scale) <= TOL
    g64 = _collide(bz, plan, fhat, dtype=torch.complex64)
    assert float(np.max(np.abs(g64 - full)) / scale) <= 2 * TOL
    f = torch.from_numpy(fhat).cuda()
    mom = bz.bz_moments(plan, f)
    assert np.allclose(mom, spectral.moments(fhat, L), rtol=1e-9, atol=1e-12)
    plan.close()


def test_padded_plan_refuses_what_it_does_not_support(bz):
    N, L = 16, 10.0
    R = bi.R_from_L(L)
    plan = _padded_plan(bz, N, L, R, 0.0, 0.5, 1, 12)
    f = torch.from_numpy(bi.random_mixture(N, L, seed=9)).cuda()
    for call in (lambda: bz.bz_step_rk(plan, f, 0.0, 0.01, 1),
                 lambda: bz.bz_batch_create(plan, 2, 0),
                 lambda: bz.bz_collide_noalloc(plan, f, torch.empty_like(f))):
        with pytest.raises(bz.BzError) as e:
            call()
        assert "UNSUPPORTED" in str(e.value) or "not supported" in str(e.value)
    plan.close()
    with pytest.raises(bz.BzError):                      # padded N = 64 would need a 128 grid
        _padded_plan(bz, 64, L, R, 0.0, 0.5, 1, 12)


def test_padded_and_circular_against_exact_bkw(bz):
    """Both forms against the exact BKW operator (eq. QQ = d/dt of eq. BKW) at N = 16: the
    padded (Galerkin) form is at least as accurate as the circular one on this resolved profile."""
    N = 16
    R = 6.0
    L = bi.L_from_R(R)
    K = bi.bkw_K(6.5)
    fhat = bi.bkw_fhat(N, L, K)
    pc = bz.bz_plan_create(N, L, R, 0.0, 0.5, 8, 12)
    pp = _padded_plan(bz, N, L, R, 0.0, 0.5, 8, 12)
    exact = spectral.bkw_Q(spectral.grid_v2(N, L), K)
    errs = {}
    for name, plan in [("circular", pc), ("padded", pp)]:
        Q = _collide(bz, plan, fhat)
        errs[name] = float(np.max(np.abs(spectral.to_grid(Q, L) - exact)))
    print(f"BKW N=16 max error vs exact: circular {errs['circular']:.3e}, padded {errs['padded']:.3e}")
    assert errs["padded"] <= 1.05 * errs["circular"]
    pc.close()
    pp.close()
