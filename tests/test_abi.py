"""The C ABI library builds, loads and exports every function that include/*.h declares (CPU only)."""
import ctypes
import math
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(bz_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    return __graft_entry__._libbuild().build()


def test_header_declares_functions():
    assert "bz_collide" in _declared() and "bz_plan_create" in _declared()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_argument_checks_without_gpu(libpath):
    import paper_2004_11239_gb300 as bz
    assert bz.bz_status_str(0) == "ok"
    assert bz.bz_status_str(1) == "invalid argument"
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    assert bz.lib.bz_plan_create(ctypes.byref(h), 20, 10.0, 9.0, 0.0, 0.5, 4, 12) == 1   # N = 20
    assert bz.lib.bz_plan_create(ctypes.byref(h), 16, -1.0, 9.0, 0.0, 0.5, 4, 12) == 1   # L < 0
    assert bz.lib.bz_collide(None, None, None, 0, None) == 1
    assert h.value is None


def test_precision_checks_without_gpu(libpath):
    """The split-BF16 form exists for the fused N = 32 pipeline only, the padded form for
    N <= 32 in FP32; the checks come before any CUDA call."""
    import paper_2004_11239_gb300 as bz
    h = ctypes.c_void_p()
    P, C = bz.BZ_CONV_PADDED, bz.BZ_CONV_CIRCULAR
    for N, prec, pipe, conv, want in [(16, bz.BZ_PREC_BF16X3, 0, C, 7), (32, bz.BZ_PREC_BF16X3, bz.BZ_PIPE_CHUNKED, C, 7),
                                      (32, 5, 0, C, 1), (64, 0, 0, P, 7), (16, bz.BZ_PREC_BF16X3, 0, P, 7),
                                      (16, 0, 0, 5, 1)]:
        d = bz.bz_plan_desc()
        d.N, d.L, d.R, d.gamma, d.s, d.N_rho, d.M = N, 10.0, 9.0, 0.0, 0.5, 2, 12
        d.precision, d.pipeline, d.conv = prec, pipe, conv
        assert bz.lib.bz_plan_create_ex(ctypes.byref(h), ctypes.byref(d)) == want
        assert h.value is None
    # CTAs per SM: 3 only for the real-data form at N = 32
    for N, data, ctas, hp, want in [(32, 0, 3, 0, 7), (16, 1, 3, 0, 7), (16, 1, 3, 2, 7), (32, 1, 4, 0, 7)]:
        d = bz.bz_plan_desc()
        d.N, d.L, d.R, d.gamma, d.s, d.N_rho, d.M = N, 10.0, 9.0, 0.0, 0.5, 2, 12
        d.data, d.ctas_per_sm, d.h_precision = data, ctas, hp
        assert bz.lib.bz_plan_create_ex(ctypes.byref(h), ctypes.byref(d)) == want
        assert h.value is None
    # the real-data form: 3D FP32 circular, M even; the fused pipeline only where N divides 32
    for N, M, prec, pipe, data, want in [(32, 12, 0, 0, 2, 1), (32, 12, bz.BZ_PREC_BF16X3, 0, 1, 7), (32, 9, 0, 0, 1, 7),
                                         (48, 12, 0, bz.BZ_PIPE_FUSED, 1, 7), (24, 12, 0, bz.BZ_PIPE_FUSED, 1, 7)]:
        d = bz.bz_plan_desc()
        d.N, d.L, d.R, d.gamma, d.s, d.N_rho, d.M = N, 10.0, 9.0, 0.0, 0.5, 2, M
        d.precision, d.pipeline, d.data = prec, pipe, data
        assert bz.lib.bz_plan_create_ex(ctypes.byref(h), ctypes.byref(d)) == want
        assert h.value is None


def test_transport_checks_without_gpu(libpath):
    """bz_transport_x validates its arguments before any CUDA call."""
    import paper_2004_11239_gb300 as bz
    dummy = ctypes.c_void_p(16)
    for N, L, nx, Lx, dt, t, want in [(12, 6.0, 8, 3.0, 1, 0.1, 7), (16, 6.0, 64, 3.0, 1, 0.1, 7), (16, 6.0, 8, -1.0, 1, 0.1, 1),
                                      (16, 0.0, 8, 3.0, 1, 0.1, 1), (16, 6.0, 8, 3.0, 5, 0.1, 1),
                                      (16, 6.0, 8, 3.0, 1, float("nan"), 1)]:
        assert bz.lib.bz_transport_x(N, L, nx, Lx, dummy, dt, t, None) == want
    assert bz.lib.bz_inhom_step(None, 8, 3.0, dummy, 1, 0.1, 1, None) == 1


@pytest.mark.parametrize("N_rho,M,gamma", [(16, 12, 0.0), (32, 32, -1.0), (5, 72, -2.0), (8, 64, 0.5)])
def test_library_quadrature_matches_oracle(libpath, N_rho, M, gamma):
    """The library's host quadrature (Newton Gauss-Legendre, its own sphere rules) equals the oracle's."""
    import numpy as np
    import paper_2004_11239_gb300 as bz
    from oracle import quadrature
    R = 6.0
    r, wr, q, wq, c = bz.bz_quadrature(N_rho, R, M, gamma)
    r2, wr2, q2, wq2 = quadrature.terms(N_rho, R, M)
    assert np.allclose(r, r2, rtol=0, atol=1e-13 * R)
    assert np.allclose(wr, wr2, rtol=1e-12)
    assert np.allclose(q, q2, rtol=0, atol=1e-14)
    assert np.allclose(wq, wq2, rtol=1e-13)
    assert np.allclose(c, wr2 * wq2 * r2 ** (gamma + 2), rtol=1e-12)


@pytest.mark.parametrize("name,kid,s", [("family", 0, 0.0), ("family", 0, 0.25), ("family", 0, 0.5),
                                        ("family", 0, 0.75), ("b5", 1, 0.0), ("b8", 2, 0.0)])
def test_library_kernel_constants_match_oracle(libpath, name, kid, s):
    import paper_2004_11239_gb300 as bz
    from oracle import kernels
    k = kernels.Kernel(name, s)
    c, A = bz.bz_kernel_constants(kid, s)
    assert abs(c - k.c) <= 1e-14 * k.c
    for got, ref in zip(A, k.taylor_moments(math.pi / 1000)):
        assert abs(got - ref) <= 1e-11 * abs(ref)


def test_library_rejects_unknown_sphere_rule(libpath):
    import paper_2004_11239_gb300 as bz
    with pytest.raises(bz.BzError):
        bz.bz_quadrature(4, 6.0, 13, 0.0)
    with pytest.raises(bz.BzError):
        bz.bz_kernel_constants(0, 1.5)


def test_checkpoint_file_checks_without_gpu(libpath, tmp_path):
    import paper_2004_11239_gb300 as bz
    with pytest.raises(bz.BzError) as e:
        bz.bz_checkpoint_plan_desc(str(tmp_path / "missing.bzck"))
    assert e.value.code == 1
    junk = tmp_path / "junk.bzck"
    junk.write_bytes(b"not a checkpoint at all" * 10)
    with pytest.raises(bz.BzError) as e:
        bz.bz_checkpoint_plan_desc(str(junk))
    assert e.value.code == 1
    assert bz.lib.bz_plan_wait_selftest(None, 100, None) == 1
    assert bz.lib.bz_plan_check_finite(None, None) == 1
