"""Host logic of bench.py's oracle legs (CPU): the term ranges, the oracle spread over
processes, and the sampled-mode error, on a small operator."""
import numpy as np

import bench
import bz_inputs as bi
from oracle import kernels, spectral


def test_split_covers_the_range_in_order():
    for p0, p1, parts in ((0, 1024, 16), (3, 17, 5), (0, 7, 7)):
        r = bench._split(p0, p1, parts)
        assert r[0][0] == p0 and r[-1][1] == p1
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1


def test_oracle_cores_and_sampled_error_match_the_oracle():
    """The collide summed over per-process term ranges equals the oracle's collide, and the
    sampled-mode error of the oracle's own result is at rounding level."""
    w = dict(N=8, N_rho=3, M=12, gamma=-1.0, s=0.5)
    L = 6.0
    R = bi.R_from_L(L)
    f = bi.random_mixture(8, L, seed=9, box=1.5)
    plan = spectral.OraclePlan(8, L, R, -1.0, kernels.Kernel("family", 0.5), 3, 12)
    full = spectral.collide_real(plan, f)
    oc = bench.OracleCores(bench._oracle_spec(w, L, R), bench._split(0, 36, 3))
    try:
        oc.build()
        q, _ = oc.collide(f, True)
    finally:
        oc.close()
    assert np.max(np.abs(q - full)) < 1e-13 * np.max(np.abs(full))
    e = bench.error_vs_oracle(w, L, R, f, full, real=True, also_realq=True)
    assert e["rel_linf"] < 1e-12
    assert e["rel_linf_vs_eq_realQ"] > 1e-6          # the real band differs from eq. realQ on this f
    e2 = bench.error_vs_oracle(w, L, R, f, spectral.collide(plan, f, 6, 20), p0=6, p1=20)
    assert e2["rel_linf"] < 1e-12
