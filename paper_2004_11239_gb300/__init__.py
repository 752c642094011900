"""Python binding of libbz (include/bz.h): argument marshalling only.

Every computation runs in the CUDA library; importing this module raises if the
built library is missing.  Device arrays are torch tensors (complex64 or
complex128, contiguous, on the plan's device); streams are torch.cuda.Stream
objects (None = the current stream).

Functions mirror the C names: bz_plan_create, bz_plan_create_ex, bz_plan_destroy,
bz_plan_info, bz_plan_terms, bz_collide, bz_collide_terms, bz_step_rk, bz_moments,
bz_ftable_entries, bz_plan_alpha, bz_plan_last_launches, bz_status_str.
"""
from __future__ import annotations

import ctypes
import math
import os

__all__ = [
    "BZ_C64", "BZ_C128", "BZ_KERNEL_FAMILY", "BZ_KERNEL_B5", "BZ_KERNEL_B8", "BzError",
    "bz_plan_create", "bz_plan_create_ex", "bz_plan_destroy", "bz_plan_info", "bz_plan_terms",
    "bz_collide", "bz_collide_terms", "bz_step_rk", "bz_moments", "bz_ftable_entries",
    "bz_plan_alpha", "bz_plan_last_launches", "bz_plan_device_errors", "bz_status_str", "library_path", "lib",
    "bz_plan_set_timing", "bz_plan_timing", "bz_collide_noalloc", "bz_plan_pipeline",
    "bz_quadrature", "bz_kernel_constants", "bz_partition_terms", "bz_plan_check_finite",
    "bz_plan_wait_selftest", "bz_checkpoint_write", "bz_checkpoint_plan_desc", "bz_checkpoint_read",
    "bz_plan_create_from_desc",
    "bz_batch_create", "bz_batch_destroy", "bz_batch_set_gamma", "bz_batch_collide", "bz_batch_step_rk",
    "bz_batch_last_launches", "bz_server_create", "bz_submit", "bz_poll", "bz_server_stats",
    "bz_transport_x", "bz_inhom_step", "bz_plan_kernel",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libbz.so")

BZ_C64, BZ_C128 = 0, 1
BZ_KERNEL_FAMILY, BZ_KERNEL_B5, BZ_KERNEL_B8 = 0, 1, 2
BZ_KERNEL_B1, BZ_KERNEL_B2, BZ_KERNEL_B3, BZ_KERNEL_B4 = 3, 4, 5, 6   # 2D kernels (dim = 2)
BZ_KERNEL_DEBYE = 7                                                     # 3D Debye-Yukawa (use gamma = 1)
BZ_PREC_FP32, BZ_PREC_BF16X3 = 0, 1
BZ_PIPE_AUTO, BZ_PIPE_FUSED, BZ_PIPE_CHUNKED = 0, 1, 2
BZ_H_AUTO, BZ_H_FP64, BZ_H_FP32 = 0, 1, 2
BZ_CONV_CIRCULAR, BZ_CONV_PADDED = 0, 1
BZ_DATA_COMPLEX, BZ_DATA_REAL = 0, 1
_STATUS = {0: "BZ_OK", 1: "BZ_ERR_ARG", 2: "BZ_ERR_OOM", 3: "BZ_ERR_CUDA", 4: "BZ_ERR_TIMEOUT",
           5: "BZ_ERR_NONFINITE", 6: "BZ_ERR_BUSY", 7: "BZ_ERR_UNSUPPORTED"}


class bz_request(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_double), ("R", ctypes.c_double),
                ("gamma", ctypes.c_double), ("s", ctypes.c_double), ("N_rho", ctypes.c_int),
                ("M", ctypes.c_int), ("kernel", ctypes.c_int), ("fhat0", ctypes.c_void_p),
                ("dtype", ctypes.c_int), ("t0", ctypes.c_double), ("t_end", ctypes.c_double),
                ("dt", ctypes.c_double), ("max_queue_s", ctypes.c_double), ("data", ctypes.c_int),
                ("precision", ctypes.c_int)]


class bz_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("steps", ctypes.c_int), ("t", ctypes.c_double),
                ("latency_s", ctypes.c_double), ("queue_s", ctypes.c_double)]


class BzError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {_STATUS.get(code, code)}")
        self.code = code


class bz_plan_desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_double), ("R", ctypes.c_double),
                ("gamma", ctypes.c_double), ("s", ctypes.c_double), ("N_rho", ctypes.c_int),
                ("M", ctypes.c_int), ("kernel", ctypes.c_int), ("precision", ctypes.c_int),
                ("eps", ctypes.c_double), ("sphere_xyz", ctypes.POINTER(ctypes.c_double)),
                ("sphere_w", ctypes.POINTER(ctypes.c_double)), ("chunk_terms", ctypes.c_int),
                ("pipeline", ctypes.c_int), ("cluster", ctypes.c_int), ("h_precision", ctypes.c_int),
                ("conv", ctypes.c_int), ("dim", ctypes.c_int), ("theta0", ctypes.c_double),
                ("data", ctypes.c_int), ("ctas_per_sm", ctypes.c_int)]


def library_path() -> str:
    return _LIB_PATH


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libbz.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(_LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    c_int, c_double, c_size = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "bz_plan_create": [ctypes.POINTER(vp), c_int, c_double, c_double, c_double, c_double, c_int, c_int],
        "bz_plan_create_ex": [ctypes.POINTER(vp), ctypes.POINTER(bz_plan_desc)],
        "bz_plan_info": [vp, ip, ctypes.POINTER(c_size), ctypes.POINTER(c_size)],
        "bz_plan_terms": [vp, dp, dp, dp, dp, dp],
        "bz_plan_pipeline": [vp, ip, ip, ip, ctypes.POINTER(ctypes.c_float)],
        "bz_quadrature": [c_int, c_double, c_int, c_double, dp, dp, dp, dp, dp],
        "bz_kernel_constants": [c_int, c_double, c_double, dp, dp],
        "bz_partition_terms": [c_int, c_int, c_int, c_int, ip, ip],
        "bz_plan_check_finite": [vp, ip],
        "bz_plan_wait_selftest": [vp, ctypes.c_longlong, vp],
        "bz_checkpoint_write": [vp, vp, c_int, c_double, ctypes.c_char_p, vp],
        "bz_checkpoint_plan_desc": [ctypes.c_char_p, ctypes.POINTER(bz_plan_desc), dp],
        "bz_checkpoint_read": [vp, ctypes.c_char_p, vp, c_int, dp, vp],
        "bz_collide": [vp, vp, vp, c_int, vp],
        "bz_collide_terms": [vp, c_int, c_int, vp, vp, c_int, vp],
        "bz_step_rk": [vp, vp, c_int, dp, c_double, c_int, vp, vp],
        "bz_moments": [vp, vp, c_int, dp, vp],
        "bz_ftable_entries": [vp, c_int, vp, vp, vp],
        "bz_plan_alpha": [vp, c_int, c_int, vp, vp],
        "bz_collide_noalloc": [vp, vp, vp, c_int, vp],
        "bz_plan_device_errors": [vp, ip],
        "bz_batch_create": [ctypes.POINTER(vp), vp, c_int, c_int],
        "bz_batch_info": [vp, ip, ip, ctypes.POINTER(c_size)],
        "bz_batch_set_gamma": [vp, c_int, c_double],
        "bz_batch_collide": [vp, c_int, ip, vp, vp, c_int, vp],
        "bz_batch_step_rk": [vp, c_int, ip, vp, c_int, c_double, c_int, vp],
        "bz_transport_x": [c_int, c_double, c_int, c_double, vp, c_int, c_double, vp],
        "bz_plan_kernel": [vp],
        "bz_inhom_step": [vp, c_int, c_double, vp, c_int, c_double, c_int, vp],
        "bz_server_create": [ctypes.POINTER(vp), c_size, c_int, c_int],
        "bz_submit": [vp, ctypes.POINTER(bz_request), ctypes.POINTER(ctypes.c_uint64)],
        "bz_poll": [vp, ctypes.c_uint64, ctypes.POINTER(bz_result), vp, c_int],
        "bz_server_stats": [vp, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long),
                            ctypes.POINTER(c_size), ip, ip],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = c_int
    L.bz_plan_set_timing.argtypes = [vp, c_int]
    L.bz_plan_set_timing.restype = c_int
    L.bz_plan_timing.argtypes = [vp, c_int, ctypes.POINTER(ctypes.c_long), dp]
    L.bz_plan_timing.restype = c_int
    L.bz_server_destroy.argtypes = [vp]
    L.bz_server_destroy.restype = None
    L.bz_batch_destroy.argtypes = [vp]
    L.bz_batch_destroy.restype = None
    L.bz_batch_last_launches.argtypes = [vp]
    L.bz_batch_last_launches.restype = c_int
    L.bz_plan_destroy.argtypes = [vp]
    L.bz_plan_destroy.restype = None
    L.bz_plan_last_launches.argtypes = [vp]
    L.bz_plan_last_launches.restype = c_int
    L.bz_status_str.argtypes = [c_int]
    L.bz_status_str.restype = ctypes.c_char_p
    L.bz_plan_kernel.argtypes = [vp]
    L.bz_plan_kernel.restype = ctypes.c_char_p
    return L


lib = _load()


def _check(code: int, what: str):
    if code != 0:
        raise BzError(code, what)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype(t) -> int:
    import torch
    if t.dtype == torch.complex64:
        return BZ_C64
    if t.dtype == torch.complex128:
        return BZ_C128
    raise TypeError(f"unsupported dtype {t.dtype}")


def _dev(t, n3: int):
    if not t.is_cuda or not t.is_contiguous() or t.numel() != n3:
        raise ValueError(f"expected a contiguous CUDA tensor of {n3} complex values (N^d)")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """Owning handle of a bz_plan (destroyed with the object or by close())."""

    def __init__(self, handle: ctypes.c_void_p, N: int, L: float, dim: int = 3, data: int = BZ_DATA_COMPLEX):
        self.handle = handle
        self.N = N
        self.L = L
        self.dim = dim
        self.data = data
        P = ctypes.c_int()
        ab = ctypes.c_size_t()
        wb = ctypes.c_size_t()
        _check(lib.bz_plan_info(handle, ctypes.byref(P), ctypes.byref(ab), ctypes.byref(wb)), "bz_plan_info")
        self.P, self.alpha_bytes, self.workspace_bytes = P.value, ab.value, wb.value

    @property
    def n3(self) -> int:
        """Modes of one field: N^3, or N^2 for a 2D plan."""
        return self.N ** self.dim

    def close(self):
        if self.handle:
            lib.bz_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bz_plan_create(N: int, L: float, R: float, gamma: float, s: float, N_rho: int, M: int) -> Plan:
    h = ctypes.c_void_p()
    _check(lib.bz_plan_create(ctypes.byref(h), N, L, R, gamma, s, N_rho, M), "bz_plan_create")
    return Plan(h, N, L)


def bz_plan_create_ex(N: int, L: float, R: float, gamma: float, s: float, N_rho: int, M: int,
                      kernel: int = BZ_KERNEL_FAMILY, eps: float = 0.0, sphere=None,
                      chunk_terms: int = 0, pipeline: int = BZ_PIPE_AUTO, cluster: int = 0,
                      h_precision: int = BZ_H_AUTO, precision: int = BZ_PREC_FP32,
                      conv: int = BZ_CONV_CIRCULAR, dim: int = 3, theta0: float = 0.0,
                      data: int = BZ_DATA_COMPLEX, ctas_per_sm: int = 0) -> Plan:
    d = bz_plan_desc()
    d.N, d.L, d.R, d.gamma, d.s, d.N_rho, d.M = N, L, R, gamma, s, N_rho, M
    d.kernel, d.precision, d.eps, d.chunk_terms = kernel, precision, eps, chunk_terms
    d.pipeline = pipeline
    d.cluster = cluster
    d.h_precision = h_precision
    d.conv = conv
    d.dim = dim
    d.theta0 = theta0
    d.data = data
    d.ctas_per_sm = ctas_per_sm
    keep = []
    if sphere is not None:
        import numpy as np
        xyz = np.ascontiguousarray(sphere[0], dtype=np.float64)
        w = np.ascontiguousarray(sphere[1], dtype=np.float64)
        keep += [xyz, w]
        d.sphere_xyz = xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.sphere_w = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    _check(lib.bz_plan_create_ex(ctypes.byref(h), ctypes.byref(d)), "bz_plan_create_ex")
    return Plan(h, N, L, dim, data)


def bz_plan_destroy(plan: Plan):
    plan.close()


def bz_plan_info(plan: Plan):
    return plan.P, plan.alpha_bytes, plan.workspace_bytes


def bz_plan_pipeline(plan: Plan):
    """{'pipeline': 'fused'|'chunked', 'cluster': C, 'clusters': G, 'tuned_ms': t}."""
    p, c, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    t = ctypes.c_float()
    _check(lib.bz_plan_pipeline(plan.handle, ctypes.byref(p), ctypes.byref(c), ctypes.byref(g), ctypes.byref(t)),
           "bz_plan_pipeline")
    return {"pipeline": "fused" if p.value == BZ_PIPE_FUSED else "chunked", "cluster": c.value,
            "clusters": g.value, "tuned_ms": t.value, "kernel": lib.bz_plan_kernel(plan.handle).decode()}


def bz_partition_terms(P: int, data: int, world: int, rank: int):
    """Host-only: the term range (p0, p1) of `rank` in a collide sharded over `world` ranks."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib.bz_partition_terms(P, data, world, rank, ctypes.byref(a), ctypes.byref(b)), "bz_partition_terms")
    return a.value, b.value


def bz_quadrature(N_rho: int, R: float, M: int, gamma: float):
    """Host-only term list: numpy arrays r, w_r, qhat[P,3], w_q, c."""
    import numpy as np
    P = N_rho * M
    r, wr, wq, c = (np.empty(P) for _ in range(4))
    q = np.empty((P, 3))
    f = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    _check(lib.bz_quadrature(N_rho, R, M, gamma, f(r), f(wr), f(q), f(wq), f(c)), "bz_quadrature")
    return r, wr, q, wq, c


def bz_kernel_constants(kernel: int, s: float, eps: float = 0.0):
    """Host-only kernel constant c and part-I moments (A1, A2, A3)."""
    c = ctypes.c_double()
    A = (ctypes.c_double * 3)()
    _check(lib.bz_kernel_constants(kernel, s, eps, ctypes.byref(c), A), "bz_kernel_constants")
    return c.value, tuple(A)


def bz_plan_terms(plan: Plan):
    """Returns numpy arrays r, w_r, qhat[P,3], w_q, c."""
    import numpy as np
    P = plan.P
    r, wr, wq, c = (np.empty(P) for _ in range(4))
    q = np.empty((P, 3))
    f = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    _check(lib.bz_plan_terms(plan.handle, f(r), f(wr), f(q), f(wq), f(c)), "bz_plan_terms")
    return r, wr, q, wq, c


def bz_collide(plan: Plan, fhat, Qhat, stream=None):
    dt = _dtype(fhat)
    if _dtype(Qhat) != dt:
        raise TypeError("fhat and Qhat must have the same dtype")
    _check(lib.bz_collide(plan.handle, _dev(fhat, plan.n3), _dev(Qhat, plan.n3), dt, _stream(stream)),
           "bz_collide")


def bz_collide_terms(plan: Plan, p0: int, p1: int, fhat, Qhat, stream=None):
    dt = _dtype(fhat)
    if _dtype(Qhat) != dt:
        raise TypeError("fhat and Qhat must have the same dtype")
    _check(lib.bz_collide_terms(plan.handle, p0, p1, _dev(fhat, plan.n3), _dev(Qhat, plan.n3), dt,
                                _stream(stream)), "bz_collide_terms")


def bz_collide_noalloc(plan: Plan, fhat, Qhat, stream=None):
    """bz_collide with its scratch in the library's fixed device array (no allocation)."""
    dt = _dtype(fhat)
    if _dtype(Qhat) != dt:
        raise TypeError("fhat and Qhat must have the same dtype")
    _check(lib.bz_collide_noalloc(plan.handle, _dev(fhat, plan.n3), _dev(Qhat, plan.n3), dt,
                                  _stream(stream)), "bz_collide_noalloc")


def bz_step_rk(plan: Plan, fhat, t: float, dt: float, nsteps: int, stream=None) -> float:
    tt = ctypes.c_double(t)
    _check(lib.bz_step_rk(plan.handle, _dev(fhat, plan.n3), _dtype(fhat), ctypes.byref(tt), dt, nsteps,
                          None, _stream(stream)), "bz_step_rk")
    return tt.value


def bz_moments(plan: Plan, fhat, stream=None):
    out = (ctypes.c_double * 5)()
    _check(lib.bz_moments(plan.handle, _dev(fhat, plan.n3), _dtype(fhat), out, _stream(stream)),
           "bz_moments")
    return list(out)


def bz_ftable_entries(plan: Plan, k_idx, term):
    """F in FP64 at device int32 tensors k_idx[E,3] (array indices) and term[E]; returns [E] complex128."""
    import torch
    E = term.numel()
    out = torch.empty(E, dtype=torch.complex128, device=term.device)
    _check(lib.bz_ftable_entries(plan.handle, E, ctypes.c_void_p(k_idx.data_ptr()),
                                 ctypes.c_void_p(term.data_ptr()), ctypes.c_void_p(out.data_ptr())),
           "bz_ftable_entries")
    return out


def bz_plan_alpha(plan: Plan, p0: int, p1: int, stream=None):
    import torch
    out = torch.empty((p1 - p0, plan.N, plan.N, plan.N), dtype=torch.complex64, device="cuda")
    _check(lib.bz_plan_alpha(plan.handle, p0, p1, ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "bz_plan_alpha")
    return out


def bz_plan_last_launches(plan: Plan) -> int:
    return lib.bz_plan_last_launches(plan.handle)


def bz_plan_device_errors(plan: Plan) -> int:
    """1 if a bounded device-side wait of the plan's kernels gave up (results invalid)."""
    c = ctypes.c_int()
    _check(lib.bz_plan_device_errors(plan.handle, ctypes.byref(c)), "bz_plan_device_errors")
    return c.value


def bz_plan_check_finite(plan: Plan) -> int:
    """1 if a result written since the last check held NaN or Inf (the flag is cleared), else 0."""
    c = ctypes.c_int()
    code = lib.bz_plan_check_finite(plan.handle, ctypes.byref(c))
    if code not in (0, 5):
        _check(code, "bz_plan_check_finite")
    return c.value


def bz_plan_wait_selftest(plan: Plan, cycles: int, stream=None):
    _check(lib.bz_plan_wait_selftest(plan.handle, int(cycles), _stream(stream)), "bz_plan_wait_selftest")


def bz_checkpoint_write(plan: Plan, fhat, t: float, path: str, stream=None):
    _check(lib.bz_checkpoint_write(plan.handle, _dev(fhat, plan.n3), _dtype(fhat), float(t), path.encode(),
                                   _stream(stream)), "bz_checkpoint_write")


def bz_checkpoint_plan_desc(path: str):
    """(bz_plan_desc, t) recorded in a checkpoint file."""
    d = bz_plan_desc()
    t = ctypes.c_double()
    _check(lib.bz_checkpoint_plan_desc(path.encode(), ctypes.byref(d), ctypes.byref(t)), "bz_checkpoint_plan_desc")
    return d, t.value


def bz_plan_create_from_desc(d: bz_plan_desc) -> Plan:
    """A plan from a filled bz_plan_desc (for example from bz_checkpoint_plan_desc)."""
    h = ctypes.c_void_p()
    _check(lib.bz_plan_create_ex(ctypes.byref(h), ctypes.byref(d)), "bz_plan_create_ex")
    return Plan(h, d.N, d.L, d.dim if d.dim else 3, d.data)


def bz_checkpoint_read(plan: Plan, path: str, fhat, stream=None) -> float:
    """Loads the checkpoint's coefficients into fhat (device tensor); returns its t."""
    t = ctypes.c_double()
    _check(lib.bz_checkpoint_read(plan.handle, path.encode(), _dev(fhat, plan.n3), _dtype(fhat), ctypes.byref(t),
                                  _stream(stream)), "bz_checkpoint_read")
    return t.value


BZ_K_PLANE_INV, BZ_K_PENCIL, BZ_K_PLANE_FWD, BZ_K_REDUCE, BZ_K_OTHER = range(5)
KERNEL_KINDS = {"plane_inv": 0, "pencil": 1, "plane_fwd": 2, "reduce": 3, "other": 4, "fused": 5}


def bz_plan_set_timing(plan: Plan, max_launches: int):
    _check(lib.bz_plan_set_timing(plan.handle, max_launches), "bz_plan_set_timing")


def bz_plan_timing(plan: Plan, kind: int):
    """(launches, total milliseconds) for one kernel kind since bz_plan_set_timing."""
    n = ctypes.c_long()
    ms = ctypes.c_double()
    _check(lib.bz_plan_timing(plan.handle, kind, ctypes.byref(n), ctypes.byref(ms)), "bz_plan_timing")
    return n.value, ms.value


class Batch:
    """Owning handle of a bz_batch (keeps its plan alive)."""

    def __init__(self, handle, plan: Plan):
        self.handle = handle
        self.plan = plan
        cap, tb = ctypes.c_int(), ctypes.c_int()
        wb = ctypes.c_size_t()
        _check(lib.bz_batch_info(handle, ctypes.byref(cap), ctypes.byref(tb), ctypes.byref(wb)), "bz_batch_info")
        self.capacity, self.terms_per_item, self.workspace_bytes = cap.value, tb.value, wb.value

    def close(self):
        if self.handle:
            lib.bz_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _slots(slots):
    arr = (ctypes.c_int * len(slots))(*[int(x) for x in slots])
    return len(slots), arr


def bz_batch_create(plan: Plan, capacity: int, terms_per_item: int = 0) -> Batch:
    h = ctypes.c_void_p()
    _check(lib.bz_batch_create(ctypes.byref(h), plan.handle, capacity, terms_per_item), "bz_batch_create")
    return Batch(h, plan)


def bz_batch_destroy(batch: Batch):
    batch.close()


def bz_batch_set_gamma(batch: Batch, slot: int, gamma: float):
    _check(lib.bz_batch_set_gamma(batch.handle, slot, gamma), "bz_batch_set_gamma")


def _dev_batch(t, batch: Batch):
    n = batch.capacity * batch.plan.n3
    if not t.is_cuda or not t.is_contiguous() or t.numel() != n:
        raise ValueError("expected a contiguous CUDA tensor of capacity * N^3 complex values")
    return ctypes.c_void_p(t.data_ptr())


def bz_batch_collide(batch: Batch, slots, fhat, Qhat, stream=None):
    n, arr = _slots(slots)
    dt = _dtype(fhat)
    if _dtype(Qhat) != dt:
        raise TypeError("fhat and Qhat must have the same dtype")
    _check(lib.bz_batch_collide(batch.handle, n, arr, _dev_batch(fhat, batch), _dev_batch(Qhat, batch), dt,
                                _stream(stream)), "bz_batch_collide")


def bz_batch_step_rk(batch: Batch, slots, fhat, dt: float, nsteps: int, stream=None):
    n, arr = _slots(slots)
    _check(lib.bz_batch_step_rk(batch.handle, n, arr, _dev_batch(fhat, batch), _dtype(fhat), dt, nsteps,
                                _stream(stream)), "bz_batch_step_rk")


def bz_batch_last_launches(batch: Batch) -> int:
    return lib.bz_batch_last_launches(batch.handle)


def _dev_cells(t, nx: int, N: int):
    if not t.is_cuda or not t.is_contiguous() or t.numel() != nx * N ** 3:
        raise ValueError(f"expected a contiguous CUDA tensor of nx * N^3 = {nx * N ** 3} complex values")
    return ctypes.c_void_p(t.data_ptr())


def bz_transport_x(N: int, L: float, nx: int, Lx: float, fcells, t: float, stream=None):
    """Free streaming of the [nx][N^3] cells over time t, in place."""
    _check(lib.bz_transport_x(N, L, nx, Lx, _dev_cells(fcells, nx, N), _dtype(fcells), t, _stream(stream)),
           "bz_transport_x")


def bz_inhom_step(batch: Batch, nx: int, Lx: float, fcells, dt: float, nsteps: int, stream=None):
    """nsteps Strang steps (free streaming, RK4 collision per cell) of the [nx][N^3] cells, in place."""
    _check(lib.bz_inhom_step(batch.handle, nx, Lx, _dev_cells(fcells, nx, batch.plan.N), _dtype(fcells), dt,
                             nsteps, _stream(stream)), "bz_inhom_step")


class Server:
    """Owning handle of a bz_server."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            lib.bz_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bz_server_create(hbm_budget_bytes: int, max_batch: int = 64, terms_per_item: int = 0) -> Server:
    h = ctypes.c_void_p()
    _check(lib.bz_server_create(ctypes.byref(h), hbm_budget_bytes, max_batch, terms_per_item), "bz_server_create")
    return Server(h)


def bz_submit(server: Server, fhat0, N: int, L: float, R: float, gamma: float, s: float, N_rho: int, M: int,
              t0: float, t_end: float, dt: float, kernel: int = BZ_KERNEL_FAMILY, max_queue_s: float = 0.0,
              data: int = BZ_DATA_COMPLEX, precision: int = BZ_PREC_FP32) -> int:
    """fhat0: host numpy array of N^3 complex128 (or complex64) coefficients; returns the ticket."""
    import numpy as np
    a = np.ascontiguousarray(fhat0)
    dt_code = BZ_C128 if a.dtype == np.complex128 else BZ_C64
    if a.dtype not in (np.complex128, np.complex64) or a.size != N ** 3:
        raise ValueError("fhat0 must hold N^3 complex64/complex128 values")
    r = bz_request(N, L, R, gamma, s, N_rho, M, kernel, a.ctypes.data, dt_code, t0, t_end, dt, max_queue_s,
                   data, precision)
    t = ctypes.c_uint64()
    _check(lib.bz_submit(server.handle, ctypes.byref(r), ctypes.byref(t)), "bz_submit")
    return t.value


def bz_poll(server: Server, ticket: int, N: int):
    """None while pending; else (bz_result, numpy complex128 coefficients or None)."""
    import numpy as np
    res = bz_result()
    out = np.empty((N, N, N), dtype=np.complex128)
    code = lib.bz_poll(server.handle, ticket, ctypes.byref(res), ctypes.c_void_p(out.ctypes.data), BZ_C128)
    if code == 6:
        return None
    _check(code, "bz_poll")
    return res, (out if res.status == 0 else None)


def bz_server_stats(server: Server):
    c, st = ctypes.c_long(), ctypes.c_long()
    u = ctypes.c_size_t()
    q, a = ctypes.c_int(), ctypes.c_int()
    _check(lib.bz_server_stats(server.handle, ctypes.byref(c), ctypes.byref(st), ctypes.byref(u), ctypes.byref(q),
                               ctypes.byref(a)), "bz_server_stats")
    return {"completed": c.value, "steps": st.value, "hbm_used": u.value, "queued": q.value, "active": a.value}


def bz_status_str(code: int) -> str:
    return lib.bz_status_str(code).decode()


def default_R(L: float) -> float:
    """R from L = (3 + sqrt 2) R / 4 (Sec. 2 anti-aliasing bound with R = 2S)."""
    return 4.0 * L / (3.0 + math.sqrt(2.0))
