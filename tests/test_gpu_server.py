"""Serving loop (bz_server_*): results alone and in a concurrent mix, against the oracle (GPU)."""
import time

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


def _wait(bz, server, tickets, Ns, timeout=600.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t, N in zip(tickets, Ns):
            if t in out:
                continue
            r = bz.bz_poll(server, t, N)
            if r is not None:
                out[t] = r
        assert time.time() - t0 < timeout, "requests did not finish"
        time.sleep(0.005)
    return [out[t] for t in tickets]


R = 6.0
L = bi.L_from_R(R)


def _req(N, gamma, s, N_rho, M, f, t_end=6.6, dt=0.025):
    return dict(fhat0=f, N=N, L=L, R=R, gamma=gamma, s=s, N_rho=N_rho, M=M, t0=6.5, t_end=t_end, dt=dt)


def test_result_alone_equals_result_in_the_mix_and_matches_oracle(bz):
    fA = bi.bkw_fhat(16, L, bi.bkw_K(6.5))
    server = bz.bz_server_create(16 << 30, max_batch=8, terms_per_item=8)
    ta = bz.bz_submit(server, **_req(16, 0.0, 0.5, 4, 12, fA))
    (resA, outA), = _wait(bz, server, [ta], [16])
    assert resA.status == 0 and resA.steps == 4 and abs(resA.t - 6.6) < 1e-12
    # the same request among others of the same and of other groups, submitted together
    mix = [
        _req(16, 0.0, 0.5, 4, 12, fA),                                        # A again
        _req(16, -1.0, 0.5, 4, 12, bi.random_mixture(16, L, seed=2, box=1.0)),  # same group
        _req(24, 0.0, 0.25, 3, 12, bi.random_mixture(24, L, seed=3, box=1.0)),  # another group
        _req(16, 0.0, 0.5, 4, 12, bi.random_mixture(16, L, seed=4, box=1.0), t_end=6.55),
        _req(48, -1.0, 0.5, 1, 12, bi.random_mixture(48, L, seed=5, box=1.0), t_end=6.55),
        _req(16, -2.0, 0.5, 4, 12, bi.random_mixture(16, L, seed=6, box=1.0), dt=0.0125, t_end=6.55),
    ]
    tickets = [bz.bz_submit(server, **r) for r in mix]
    res = _wait(bz, server, tickets, [r["N"] for r in mix])
    for (rr, out), r in zip(res, mix):
        assert rr.status == 0, rr.status
        assert rr.steps == round((r["t_end"] - 6.5) / r["dt"])
    outA2 = res[0][1]
    assert np.array_equal(outA2, outA)                 # identical bits alone and in the mix
    # A against the oracle's RK4
    op = spectral.OraclePlan(16, L, R, 0.0, kernels.Kernel("family", 0.5), 4, 12)
    ref = spectral.rk4(op, fA, 0.025, 4)
    err = float(np.max(np.abs((outA - fA) - (ref - fA))) / np.max(np.abs(ref - fA)))
    print(f"served RK4: rel_Linf of the change={err:.2e}")
    assert err <= TOL
    # the N = 48 request (chunked pipeline, gamma per slot of the group's batch) equals the same
    # batch call made directly, bit for bit, and a plan built with its gamma within the bar
    r48 = mix[4]
    plan = bz.bz_plan_create(48, L, R, 0.0, 0.5, 1, 12)
    batch = bz.bz_batch_create(plan, 1, 0)
    bz.bz_batch_set_gamma(batch, 0, -1.0)
    f48 = torch.from_numpy(r48["fhat0"]).cuda().reshape(1, 48, 48, 48).contiguous()
    for _ in range(2):
        bz.bz_batch_step_rk(batch, [0], f48, 0.025, 1)
    torch.cuda.synchronize()
    assert np.array_equal(res[4][1], f48[0].cpu().numpy())
    batch.close()
    pg = bz.bz_plan_create(48, L, R, -1.0, 0.5, 1, 12)
    fg = torch.from_numpy(r48["fhat0"]).cuda()
    bz.bz_step_rk(pg, fg, 6.5, 0.025, 2)
    torch.cuda.synchronize()
    d0 = fg.cpu().numpy() - r48["fhat0"]
    assert float(np.max(np.abs(res[4][1] - r48["fhat0"] - d0)) / np.max(np.abs(d0))) <= TOL
    pg.close()
    st = bz.bz_server_stats(server)
    assert st["completed"] == 7 and st["queued"] == 0 and st["active"] == 0
    plan.close()
    server.close()


def test_request_larger_than_the_budget_fails_cleanly(bz):
    server = bz.bz_server_create(1 << 20, max_batch=4)            # 1 MiB: no plan fits
    t = bz.bz_submit(server, **_req(16, 0.0, 0.5, 4, 12, bi.bkw_fhat(16, L, bi.bkw_K(6.5))))
    (res, out), = _wait(bz, server, [t], [16], timeout=60)
    assert res.status == 2 and out is None                        # BZ_ERR_OOM
    with pytest.raises(bz.BzError):
        bz.bz_poll(server, t, 16)                                 # ticket forgotten after the poll
    server.close()


def test_real_data_and_split_bf16_requests_alone_and_in_the_mix(bz):
    """The real-data form (batched at N = 16, per request at N = 24) and the split-BF16 form
    (N = 32) in the server: identical bits alone and in a mix of groups, and within their bars
    of the oracle's RK4 (real-data reading for the real form)."""
    fR = bi.random_mixture(16, L, seed=11, box=1.0)
    fB = bi.random_mixture(32, L, seed=12, box=1.0)
    rR = dict(_req(16, -1.0, 0.5, 4, 12, fR, t_end=6.55), data=bz.BZ_DATA_REAL)
    rB = dict(_req(32, 0.0, 0.5, 2, 32, fB, t_end=6.55), precision=bz.BZ_PREC_BF16X3)
    rC = dict(_req(24, 0.0, 0.25, 3, 12, bi.random_mixture(24, L, seed=13, box=1.0), t_end=6.55),
              data=bz.BZ_DATA_REAL)
    server = bz.bz_server_create(32 << 30, max_batch=4, terms_per_item=8)
    alone = [_wait(bz, server, [bz.bz_submit(server, **r)], [r["N"]])[0] for r in (rR, rB, rC)]
    mix = [rR, rB, rC, _req(16, 0.0, 0.5, 4, 12, bi.random_mixture(16, L, seed=14, box=1.0)),
           dict(_req(16, -1.0, 0.5, 4, 12, bi.random_mixture(16, L, seed=15, box=1.0)), data=bz.BZ_DATA_REAL)]
    res = _wait(bz, server, [bz.bz_submit(server, **r) for r in mix], [r["N"] for r in mix])
    for k in range(3):
        assert alone[k][0].status == 0 and res[k][0].status == 0
        assert np.array_equal(res[k][1], alone[k][1])
    opR = spectral.OraclePlan(16, L, R, -1.0, kernels.Kernel("family", 0.5), 4, 12)
    ref = spectral.rk4_real(opR, fR, 0.025, 2)
    err = float(np.max(np.abs(alone[0][1] - ref)) / np.max(np.abs(ref - fR)))
    print(f"served real-data RK4: rel_Linf of the change={err:.2e}")
    assert err <= TOL
    opB = spectral.OraclePlan(32, L, R, 0.0, kernels.Kernel("family", 0.5), 2, 32)
    ref = spectral.rk4(opB, fB, 0.025, 2)
    err = float(np.max(np.abs(alone[1][1] - ref)) / np.max(np.abs(ref - fB)))
    print(f"served split-BF16 RK4: rel_Linf of the change={err:.2e}")
    assert err <= 1e-3
    with pytest.raises(bz.BzError) as e:                          # BF16X3 only at N = 32, complex data
        bz.bz_submit(server, **dict(_req(16, 0.0, 0.5, 4, 12, fR), precision=bz.BZ_PREC_BF16X3))
    assert e.value.code == 7
    server.close()


def test_queue_timeout_nonfinite_result_and_independent_groups(bz):
    """max_queue_s: a request whose group cannot be placed while another group holds the budget
    fails with BZ_ERR_TIMEOUT; a NaN input ends its own request with BZ_ERR_NONFINITE and not its
    neighbours; a short request of a light group finishes long before a long request of a heavy
    group (groups step independently)."""
    server = bz.bz_server_create(100 << 20, max_batch=2, terms_per_item=8)   # room for one N = 16 group
    long_req = _req(16, 0.0, 0.5, 4, 12, bi.random_mixture(16, L, seed=21, box=1.0), t_end=6.5 + 2000 * 0.025)
    other = _req(16, 0.0, 0.25, 4, 12, bi.random_mixture(16, L, seed=22, box=1.0))   # another s: another group
    ta = bz.bz_submit(server, **long_req)
    time.sleep(0.05)
    tb = bz.bz_submit(server, **dict(other, max_queue_s=0.02))
    (rb, ob), = _wait(bz, server, [tb], [16], timeout=60)
    assert rb.status == 4 and ob is None                         # BZ_ERR_TIMEOUT
    (ra, _), = _wait(bz, server, [ta], [16])
    assert ra.status == 0
    server.close()

    server = bz.bz_server_create(32 << 30, max_batch=4, terms_per_item=8)
    good = bi.random_mixture(16, L, seed=23, box=1.0)
    bad = good.copy()
    bad[0, 1, 2] = np.nan
    heavy = _req(48, -1.0, 0.5, 8, 12, bi.random_mixture(48, L, seed=24, box=1.0), t_end=6.5 + 40 * 0.025)
    # both groups warm (plans, batch, graphs) before the timed pair
    _wait(bz, server, [bz.bz_submit(server, **dict(heavy, t_end=6.525)),
                       bz.bz_submit(server, **_req(16, 0.0, 0.5, 4, 12, good, t_end=6.525))], [48, 16])
    th = bz.bz_submit(server, **heavy)
    tg = bz.bz_submit(server, **_req(16, 0.0, 0.5, 4, 12, good, t_end=6.55))
    tn = bz.bz_submit(server, **_req(16, 0.0, 0.5, 4, 12, bad, t_end=6.55))
    (rh, _), (rg, og), (rn, on) = _wait(bz, server, [th, tg, tn], [48, 16, 16])
    assert rg.status == 0 and np.all(np.isfinite(og))
    assert rn.status == 5 and on is None                          # BZ_ERR_NONFINITE
    assert rh.status == 0
    print(f"latency: N=16 (2 steps) {rg.latency_s * 1e3:.1f} ms, N=48 (40 steps) {rh.latency_s * 1e3:.1f} ms")
    assert rg.latency_s < rh.latency_s / 3
    server.close()
