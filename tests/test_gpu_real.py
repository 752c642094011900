"""Real-data form (BZ_DATA_REAL) on the GPU against the oracle's real-data reading
(`collide_real`: Hermitian part of fhat, Nyquist planes dropped).

The GPU path shares one pair of 3D transforms between terms 2q and 2q + 1 and symmetrises the
accumulated sum once per collide; the oracle evaluates every term on its own.  Bar: relative
L-infinity error 1e-5 of max|Q| (FP32 form).  Inputs are complex and unsymmetric on purpose
(random coefficients, shifted mixtures) so that the symmetrisation of the input is exercised.
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


def _real_plan(bz, N, L, R, gamma, s, N_rho, M, kernel=0, **kw):
    return bz.bz_plan_create_ex(N, L, R, gamma, s, N_rho, M, kernel=kernel, data=bz.BZ_DATA_REAL, **kw)


def _collide(bz, plan, fhat, p0=None, p1=None, dtype=torch.complex128):
    f = torch.from_numpy(np.asarray(fhat)).to("cuda", dtype=dtype)
    q = torch.empty_like(f)
    if p0 is None:
        bz.bz_collide(plan, f, q)
    else:
        bz.bz_collide_terms(plan, p0, p1, f, q)
    torch.cuda.synchronize()
    return q.cpu().numpy().astype(np.complex128)


CASES = [
    # N, gamma, s, kernel name, kernel id, N_rho, M, data, CTAs per SM (N = 32: 2 k_fused, 3 k_pair3)
    (8, 0.0, 0.5, "family", 0, 3, 12, "random", 0),
    (16, -1.0, 0.25, "family", 0, 2, 32, "mixture", 0),
    (16, 0.0, 0.0, "b5", 1, 2, 12, "random", 0),
    (32, -2.0, 0.0, "b8", 2, 2, 12, "mixture", 2),
    (32, -2.0, 0.0, "b8", 2, 2, 12, "mixture", 3),
    (32, 0.0, 0.5, "family", 0, 3, 12, "random", 2),
    (32, 0.0, 0.5, "family", 0, 3, 12, "random", 3),
]


@pytest.mark.parametrize("N,gamma,s,name,kid,N_rho,M,data,ctas", CASES)
def test_real_collide_matches_oracle(bz, N, gamma, s, name, kid, N_rho, M, data, ctas):
    L = 10.0
    R = bi.R_from_L(L)
    fhat = bi.random_fhat(N, seed=40 + N, scale=1e-3) if data == "random" else bi.random_mixture(N, L, seed=N)
    plan = _real_plan(bz, N, L, R, gamma, s, N_rho, M, kid, ctas_per_sm=ctas)
    info = bz.bz_plan_pipeline(plan)
    assert info["pipeline"] == "fused"
    if ctas:
        assert info["kernel"] == ("k_pair3" if ctas == 3 else "k_fused")
    got = _collide(bz, plan, fhat)
    ref = spectral.collide_real(spectral.OraclePlan(N, L, R, gamma, kernels.Kernel(name, s), N_rho, M), fhat)
    err = _rel(got, ref)
    print(f"real N={N} {data} gamma={gamma} {name} s={s} P={N_rho * M} {info['kernel']} C={info['cluster']} "
          f"G={info['clusters']}: rel_Linf={err:.2e}")
    assert err <= TOL
    ny = spectral.nyquist_mask(N)
    assert np.array_equal(spectral.mirror(got)[~ny], np.conj(got)[~ny])   # symmetrised exactly off S
    assert got[0, 0, 0] == 0
    plan.close()


def test_real_term_ranges_fp32_input_and_refusals(bz):
    N, L = 16, 10.0
    R = bi.R_from_L(L)
    fhat = bi.random_mixture(N, L, seed=3)
    plan = _real_plan(bz, N, L, R, 0.0, 0.5, 2, 12)
    op = spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 2, 12)
    full = spectral.collide_real(op, fhat)
    scale = np.max(np.abs(full))
    parts = []
    for p0, p1 in [(0, 10), (10, 24)]:
        got = _collide(bz, plan, fhat, p0, p1)
        err = float(np.max(np.abs(got - spectral.collide_real(op, fhat, p0, p1))) / scale)
        print(f"real terms [{p0},{p1}): error / max|Q| = {err:.2e}")
        assert err <= TOL
        parts.append(got)
    assert float(np.max(np.abs(parts[0] + parts[1] - full)) / scale) <= 2 * TOL
    assert np.all(_collide(bz, plan, fhat, 6, 6) == 0)
    got32 = _collide(bz, plan, fhat, dtype=torch.complex64)     # FP32 caller arrays
    assert _rel(got32, full) <= TOL
    f = torch.from_numpy(fhat).cuda()
    for call in (lambda: bz.bz_collide_terms(plan, 1, 10, f, torch.empty_like(f)),      # odd bound
                 lambda: bz.bz_collide_noalloc(plan, f, torch.empty_like(f))):
        with pytest.raises(bz.BzError):
            call()
    plan.close()
    for kw in (dict(precision=bz.BZ_PREC_BF16X3), dict(conv=bz.BZ_CONV_PADDED)):
        with pytest.raises(bz.BzError):
            _real_plan(bz, 32 if "precision" in kw else N, L, R, 0.0, 0.5, 2, 12, **kw)
    with pytest.raises(bz.BzError):                              # M odd: pairs would straddle radial nodes
        _real_plan(bz, N, L, R, 0.0, 0.5, 2, 9)
    with pytest.raises(bz.BzError):                              # the fused pair kernel needs N | 32
        _real_plan(bz, 24, L, R, 0.0, 0.5, 1, 12, pipeline=bz.BZ_PIPE_FUSED)


def test_real_rk4_matches_oracle(bz):
    N, R = 16, 6.0
    L = bi.L_from_R(R)
    f0 = bi.random_mixture(N, L, seed=11, box=1.5)
    plan = _real_plan(bz, N, L, R, 0.0, 0.5, 3, 12)
    f = torch.from_numpy(f0.copy()).cuda()
    t = bz.bz_step_rk(plan, f, 0.0, 0.1, 3)
    torch.cuda.synchronize()
    assert abs(t - 0.3) < 1e-12
    op = spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 3, 12)
    ref = spectral.rk4_real(op, f0, 0.1, 3)
    err = _rel(f.cpu().numpy() - f0, ref - f0)
    print(f"real RK4 3 steps: rel_Linf of the change = {err:.2e}")
    assert err <= TOL
    plan.close()


def _summand_scale(oplan, fhat, p0, p1):
    """max_k sum_p |alpha_p(k)| max|h| max|g_p| over terms [p0, p1) of the real band: the scale
    the FP32 rounding of the summands grows with (a large shift r qhat leaves a term sum far
    below its summands)."""
    fb = spectral.real_band(fhat)
    hm = np.max(np.abs(spectral.dft3(fb, +1)))
    tot = 0.0
    for p in range(p0, p1):
        tot = tot + np.abs(oplan.alpha(p)) * hm * np.max(np.abs(spectral.dft3(fb * oplan.beta(p), +1)))
    return float(np.max(tot))


@pytest.mark.parametrize("ctas", [2, 3])
def test_real_form_at_full_size(bz, ctas):
    """The bench's workload (N = 32, P = 1024, BKW at t = 6.5; Nyquist content 5e-8 of fhat_0):
    the whole real-data collide against the oracle's reading and against the circular operator
    itself (eq. realQ on fhat as given: the real form drops only the Nyquist content of f);
    sampled term ranges (radial extremes) against the oracle relative to their summands, no
    worse than the complex form on the same terms."""
    N, R = 32, 6.0
    L = bi.L_from_R(R)
    fhat = bi.bkw_fhat(N, L, bi.bkw_K(6.5))
    pr = _real_plan(bz, N, L, R, 0.0, 0.5, 32, 32, ctas_per_sm=ctas)
    pc = bz.bz_plan_create(N, L, R, 0.0, 0.5, 32, 32)
    assert bz.bz_plan_pipeline(pr)["kernel"] == ("k_pair3" if ctas == 3 else "k_fused")
    gr = _collide(bz, pr, fhat)
    gc = _collide(bz, pc, fhat)
    op = spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 32, 32)
    err = _rel(gr, spectral.collide_real(op, fhat))
    err_c = _rel(gr, spectral.collide(op, fhat))
    print(f"real ({ctas} CTAs/SM) N=32 P=1024 BKW: rel_Linf={err:.2e} vs the real-data reading, {err_c:.2e} vs eq. realQ; "
          f"vs the complex FP32 form {_rel(gr, gc):.2e}")
    assert err <= TOL and err_c <= TOL
    for p0 in (0, 500, 1014):
        p1 = p0 + 10
        got = _collide(bz, pr, fhat, p0, p1)
        e_real = float(np.max(np.abs(got - spectral.collide_real(op, fhat, p0, p1))))
        e_cplx = float(np.max(np.abs(_collide(bz, pc, fhat, p0, p1) - spectral.collide(op, fhat, p0, p1))))
        scale = _summand_scale(op, fhat, p0, p1)
        print(f"real N=32 terms [{p0},{p1}): err/summand scale={e_real / scale:.2e} "
              f"(complex form {e_cplx / scale:.2e})")
        assert e_real / scale <= TOL
    pr.close()
    pc.close()


@pytest.mark.parametrize("N,ctas", [(16, 0), (32, 2), (32, 3)])
def test_real_batch_matches_oracle_and_is_batch_invariant(bz, N, ctas):
    """Batches of a real-data plan: per-slot gamma (the radial scale of a pair's node), the
    batched collide and RK4 against the oracle's real-data reading, and the same bits alone and
    in the batch."""
    L = 10.0
    R = bi.R_from_L(L)
    plan = _real_plan(bz, N, L, R, 0.0, 0.5, 2, 12, ctas_per_sm=ctas)
    cap = 4
    batch = bz.bz_batch_create(plan, cap, 0)
    gam = {2: -1.0, 0: 0.0, 3: -2.0}
    for slot, g in gam.items():
        bz.bz_batch_set_gamma(batch, slot, g)
    f = np.stack([bi.random_mixture(N, L, seed=500 + b) for b in range(cap)])
    fd = torch.from_numpy(f).cuda()
    qd = torch.zeros_like(fd)
    bz.bz_batch_collide(batch, [2, 0, 3], fd, qd)
    torch.cuda.synchronize()
    q = qd.cpu().numpy()
    ops = {g: spectral.OraclePlan(N, L, R, g, kernels.Kernel("family", 0.5), 2, 12) for g in set(gam.values())}
    for slot, g in gam.items():
        err = _rel(q[slot], spectral.collide_real(ops[g], f[slot]))
        print(f"real batch N={N} ({bz.bz_plan_pipeline(plan)['kernel']}) slot {slot} gamma={g}: rel_Linf={err:.2e}")
        assert err <= TOL
    assert np.all(q[1] == 0)
    alone = torch.zeros_like(fd)
    bz.bz_batch_collide(batch, [3], fd, alone)
    torch.cuda.synchronize()
    assert np.array_equal(alone.cpu().numpy()[3], q[3])      # the same bits alone and in the batch
    fr = fd.clone()
    bz.bz_batch_step_rk(batch, [0, 2], fr, 0.05, 2)
    torch.cuda.synchronize()
    got = fr.cpu().numpy()
    for slot in (0, 2):
        ref = spectral.rk4_real(ops[gam[slot]], f[slot], 0.05, 2)
        err = _rel(got[slot] - f[slot], ref - f[slot])
        print(f"real batch RK4 slot {slot}: rel_Linf of the change = {err:.2e}")
        assert err <= TOL
    assert np.array_equal(got[1], f[1]) and np.array_equal(got[3], f[3])   # inactive slots untouched
    batch.close()
    plan.close()


@pytest.mark.parametrize("N,pipe", [(24, 0), (32, 2), (48, 0)])
def test_real_chunked_matches_oracle(bz, N, pipe):
    """The chunked pipeline's pair form (N = 24, 48, or on request): whole collides of a few
    terms against the oracle's real-data reading, an RK4 change, and term ranges."""
    L = 10.0
    R = bi.R_from_L(L)
    fhat = bi.random_mixture(N, L, seed=N + 7)
    plan = _real_plan(bz, N, L, R, -1.0, 0.5, 2, 12, pipeline=pipe)
    assert bz.bz_plan_pipeline(plan)["kernel"] == "chunked"
    op = spectral.OraclePlan(N, L, R, -1.0, kernels.Kernel("family", 0.5), 2, 12)
    got = _collide(bz, plan, fhat)
    err = _rel(got, spectral.collide_real(op, fhat))
    print(f"real chunked N={N} P=24: rel_Linf={err:.2e}")
    assert err <= TOL
    parts = _collide(bz, plan, fhat, 0, 10) + _collide(bz, plan, fhat, 10, 24)
    assert _rel(parts, got) <= 2 * TOL
    if N <= 32:
        f = torch.from_numpy(fhat.copy()).cuda()
        bz.bz_step_rk(plan, f, 0.0, 0.05, 1)
        torch.cuda.synchronize()
        ref = spectral.rk4_real(op, fhat, 0.05, 1)
        e = _rel(f.cpu().numpy() - fhat, ref - fhat)
        print(f"real chunked N={N} RK4: rel_Linf of the change = {e:.2e}")
        assert e <= TOL
    plan.close()


def test_real_chunked_n64_sampled_terms(bz):
    """N = 64, N_rho = M = 64 (the single-collide workload) on the chunked pair form: sampled
    term ranges against the oracle's real-data reading, relative to their summands."""
    N, L = 64, 10.0
    R = bi.R_from_L(L)
    fhat = bi.bigaussian_noise_c3(N, L)
    plan = _real_plan(bz, N, L, R, -1.0, 0.5, 64, 64)
    for p0, p1 in [(0, 2), (2046, 2050), (4094, 4096)]:
        got = _collide(bz, plan, fhat, p0, p1)
        op = spectral.OraclePlan(N, L, R, -1.0, kernels.Kernel("family", 0.5), 64, 64, terms=np.arange(p0, p1))
        ref = spectral.collide_real(op, fhat, p0, p1)
        scale = _summand_scale(op, fhat, p0, p1)
        err = float(np.max(np.abs(got - ref))) / scale
        print(f"real chunked N=64 terms [{p0},{p1}): err/summand scale={err:.2e}, rel_Linf={_rel(got, ref):.2e}")
        assert err <= TOL
    plan.close()


@pytest.mark.parametrize("N,cluster", [(16, 1), (16, 2), (32, 4), (32, 8)])
def test_real_fused_every_cluster_size(bz, N, cluster):
    """k_fused's pair form at each compiled cluster size (plan creation times them all)."""
    L = 10.0
    R = bi.R_from_L(L)
    fhat = bi.random_mixture(N, L, seed=N + cluster)
    plan = _real_plan(bz, N, L, R, 0.0, 0.5, 2, 12, cluster=cluster, ctas_per_sm=2 if N == 32 else 0)
    info = bz.bz_plan_pipeline(plan)
    assert info["kernel"] == "k_fused" and info["cluster"] == cluster
    got = _collide(bz, plan, fhat)
    err = _rel(got, spectral.collide_real(spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 2, 12), fhat))
    print(f"real k_fused N={N} C={cluster}: rel_Linf={err:.2e}")
    assert err <= TOL
    plan.close()


def test_real_fused_with_fp32_h(bz):
    """h formed in FP32 inside k_fused's item prologue from the symmetrised input (BZ_H_FP32)."""
    N, L = 16, 10.0
    R = bi.R_from_L(L)
    fhat = bi.random_mixture(N, L, seed=61)
    plan = _real_plan(bz, N, L, R, 0.0, 0.5, 2, 12, h_precision=bz.BZ_H_FP32)
    got = _collide(bz, plan, fhat)
    err = _rel(got, spectral.collide_real(spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 2, 12), fhat))
    print(f"real N={N} FP32 h: rel_Linf={err:.2e}")
    assert err <= TOL
    with pytest.raises(bz.BzError):                              # batches need h in FP64
        bz.bz_batch_create(plan, 2, 0)
    plan.close()


def test_pair_kernel_with_fp32_h(bz):
    """k_pair3 (three CTAs per SM) with h formed in FP32 by a plane and a pencil pass
    (BZ_H_FP32): the pure-FP32 real-data form at N = 32 within the FP32 bar of the oracle, and
    its RK4 step within the bar of the FP64-h form's change."""
    N = 32
    R = 6.0
    L = bi.L_from_R(R)
    fhat = bi.bkw_fhat(N, L, bi.bkw_K(6.5))
    plan = _real_plan(bz, N, L, R, 0.0, 0.5, 4, 12, h_precision=bz.BZ_H_FP32, ctas_per_sm=3)
    assert bz.bz_plan_pipeline(plan)["kernel"] == "k_pair3"
    got = _collide(bz, plan, fhat)
    op = spectral.OraclePlan(N, L, R, 0.0, kernels.Kernel("family", 0.5), 4, 12)
    err = _rel(got, spectral.collide_real(op, fhat))
    print(f"k_pair3 FP32 h: rel_Linf={err:.2e}")
    assert err <= TOL
    ref = _real_plan(bz, N, L, R, 0.0, 0.5, 4, 12, ctas_per_sm=3)
    f1 = torch.from_numpy(fhat).cuda()
    f2 = f1.clone()
    bz.bz_step_rk(plan, f1, 6.5, 0.05, 2)
    bz.bz_step_rk(ref, f2, 6.5, 0.05, 2)
    torch.cuda.synchronize()
    d1 = f1.cpu().numpy() - fhat
    d2 = f2.cpu().numpy() - fhat
    assert _rel(d1, d2) <= TOL
    ref.close()
    plan.close()
