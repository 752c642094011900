"""Parity at the benchmark's full sizes, in the launch configuration bench.py times (GPU).

* N = 32, N_rho = 32, M = 32 (P = 1024), gamma = 0, s = 1/2, R = 6, BKW data at t = 6.5:
  the whole collide against the oracle (the oracle builds its full F table).
* N = 64, N_rho = 64, M = 64 (P = 4096), gamma = -1, s = 1/2, L = 10, bi-Gaussian + noise:
  sampled terms through bz_collide_terms against the oracle restricted to those terms,
  plus properties that hold at any size (exact mass mode, additivity over term ranges).
  A few terms are not the operator: their sum can be far smaller than its summands (a
  large shift r qhat leaves little overlap of h and g_p), while FP32 rounding scales with
  the summands.  The sampled check therefore divides the error by the summands' bound
  max_k sum_p |alpha_p(k)| max|h| max|g_p| (the full operator keeps the max|Q| bar).
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


def test_full_collide_n32_p1024_bkw(bz):
    R = 6.0
    L = bi.L_from_R(R)
    N = 32
    fhat = bi.bkw_fhat(N, L, bi.bkw_K(6.5))
    plan = bz.bz_plan_create(N, L, R, 0.0, 0.5, 32, 32)
    f = torch.from_numpy(fhat).cuda()
    q = torch.empty_like(f)
    bz.bz_collide(plan, f, q)
    torch.cuda.synchronize()
    got = q.cpu().numpy()
    oplan = spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 32, 32)
    ref = spectral.collide(oplan, fhat)
    err = _rel(got, ref)
    print(f"N=32 P=1024 BKW: rel_Linf={err:.2e}")
    assert err <= TOL
    assert got[0, 0, 0] == 0
    plan.close()


def _summand_scale(oplan, fhat, p0, p1):
    """max_k sum_p |alpha_p(k)| max|h| max|g_p|: a bound on |sum_p alpha_p Uhat_p| (|Uhat_p| <=
    max|h g_p| since Uhat_p = DFT(h g_p) / N^3), the scale FP32 rounding of the summands scales with."""
    h = spectral.dft3(fhat, +1)
    hm = np.max(np.abs(h))
    tot = 0.0
    for p in range(p0, p1):
        g = spectral.dft3(fhat * oplan.beta(p), +1)
        tot = tot + np.abs(oplan.alpha(p)) * hm * np.max(np.abs(g))
    return float(np.max(tot))


def test_sampled_terms_n64_p4096(bz):
    N, L = 64, 10.0
    R = bi.R_from_L(L)
    fhat = bi.bigaussian_noise_c3(N, L)
    plan = bz.bz_plan_create(N, L, R, -1.0, 0.5, 64, 64)
    f = torch.from_numpy(fhat).cuda()
    sel = [(0, 1), (2047, 2049), (4095, 4096)]          # radial extremes and the middle
    for p0, p1 in sel:
        q = torch.empty_like(f)
        bz.bz_collide_terms(plan, p0, p1, f, q)
        torch.cuda.synchronize()
        got = q.cpu().numpy()
        oplan = spectral.OraclePlan(N, L, R, -1.0, kernels.Kernel("family", 0.5), 64, 64,
                                    terms=np.arange(p0, p1))
        ref = spectral.collide(oplan, fhat, p0, p1)
        scale = _summand_scale(oplan, fhat, p0, p1)
        err = float(np.max(np.abs(got - ref))) / scale
        print(f"N=64 terms [{p0},{p1}): err/summand scale={err:.2e}, rel_Linf={_rel(got, ref):.2e}")
        assert err <= TOL
        assert got[0, 0, 0] == 0
    # additivity over term ranges at full size
    a, b, full = torch.empty_like(f), torch.empty_like(f), torch.empty_like(f)
    bz.bz_collide_terms(plan, 0, 1500, f, a)
    bz.bz_collide_terms(plan, 1500, 4096, f, b)
    bz.bz_collide(plan, f, full)
    torch.cuda.synchronize()
    assert _rel((a + b).cpu().numpy(), full.cpu().numpy()) <= 1e-6
    plan.close()


@pytest.mark.parametrize("data", [0, 1])
def test_whole_collide_n64_moderate_P_every_mode(bz, data):
    """A whole N = 64 collide (the bench's N = 64 data and operator, N_rho = 4, M = 12: P = 48, the full
    radial range [0, R]; two chunks, so both streams run) through the bench's chunked pipeline,
    against the oracle at every mode with the max |Qhat| bar, complex and real-data forms.  (The
    bench checks one full P = 4096 collide against the oracle at sampled modes.)"""
    N, L = 64, 10.0
    R = bi.R_from_L(L)
    fhat = bi.bigaussian_noise_c3(N, L)
    plan = bz.bz_plan_create_ex(N, L, R, -1.0, 0.5, 4, 12, data=data)
    f = torch.from_numpy(fhat).cuda()
    q = torch.empty_like(f)
    bz.bz_collide(plan, f, q)
    torch.cuda.synchronize()
    op = spectral.OraclePlan(N, L, R, -1.0, kernels.Kernel("family", 0.5), 4, 12)
    ref = (spectral.collide_real if data else spectral.collide)(op, fhat)
    err = _rel(q.cpu().numpy(), ref)
    print(f"N=64 P=48 data={data} every mode: rel_Linf={err:.2e}")
    assert err <= TOL
    plan.close()
