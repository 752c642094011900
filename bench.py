"""Throughput of the collision operator on one GB300: Q(f,f) evaluations per second.

Workload (default "rk4_n32"): the RK4 relaxation of the BKW solution, N = 32, N_rho = 32,
M = 32 (product sphere rule), gamma = 0, s = 0.5 (nu = 1), R = 6, L = (3 + sqrt 2) R / 4,
dt = 0.01, starting at t = 6.5.  One step = one RK4 step = 4 collides (P = 1024 terms each).
Inputs stay in HBM; the alpha table (268 MB) is larger than L2, so every collide streams it.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (N, N_rho, M, gamma, s, R, dt, description)
    "rk4_n32": dict(N=32, N_rho=32, M=32, gamma=0.0, s=0.5, R=6.0, dt=0.01, t0=6.5,
                    data="bkw", desc="RK4 step of the BKW solution, N=32, N_rho=32, M=32, "
                                     "gamma=0, s=0.5, R=6, L=(3+sqrt2)R/4, dt=0.01, t0=6.5"),
    "single_n64": dict(N=64, N_rho=64, M=64, gamma=-1.0, s=0.5, R=None, L=10.0, dt=None,
                       data="c3", desc="single collide, N=64, N_rho=64, M=64, gamma=-1, s=0.5, "
                                       "L=10, bi-Gaussian plus 1% noise"),
    "single_n16": dict(N=16, N_rho=16, M=12, gamma=0.0, s=0.5, R=None, L=10.0, dt=None,
                       data="c1", desc="single collide, N=16, N_rho=16, M=12, gamma=0, s=0.5, "
                                       "L=10, two Maxwellians at +-2 e1"),
    "serve": dict(N=None, N_rho=None, M=None, gamma=None, s=None, R=None, L=10.0, dt=0.02, t_end=2.0,
                  data="mixtures", desc="continuous-batching server: %d requests, Poisson arrivals at 200/s, "
                  "N in {16,24,32,48,64}, N_rho=N, M in {12,32}, gamma in {0,-1,-2}, s in {0.25,0.5}, RK4 to "
                  "t=2 (dt=0.02, 100 steps), seeded two-Maxwellian data; plans warmed before the trace"),
    "single_2d_n64": dict(N=64, N_rho=64, M=32, gamma=0.0, s=0.0, R=6.0, dt=None, data="bkw2d", dim=2,
                          kernel=6, desc="single 2D collide in the Table 1 setting: N=64, N_rho=64, M=32 circle "
                                         "points, kernel b4, R=6, L=(3+sqrt2)R/4, BKW samples at t=0"),
    "inhom_n16": dict(N=16, N_rho=16, M=12, gamma=0.0, s=0.5, R=6.0, dt=0.01, nx=32, Lx=4.0, data="inhom",
                      desc="spatially inhomogeneous df/dt + v1 df/dx = Q(f,f): 32 cells on a periodic x-interval "
                           "of length 4, N=16, N_rho=16, M=12 (icosahedron), gamma=0, s=0.5, R=6, L=(3+sqrt2)R/4; "
                           "one Strang step (free streaming dt/2, RK4 collision in every cell, free streaming dt/2) "
                           "per bench step, dt=0.01; density wave on a two-stream profile"),
    "batch_4096": dict(N=None, N_rho=None, M=32, gamma=None, s=None, R=None, L=10.0, dt=0.01,
                       data="mixtures", desc="4096 instances (3072 at N=16, 1024 at N=32), N_rho=N, "
                       "M=32, gamma in {0,-1}, s in {0.25,0.5,0.75}, two-Maxwellian mixtures, "
                       "one RK4 step per bench step; grouped by (N, s) into batches"),
}
METRIC = "Q(f,f) evals/s"


def _geometry(w):
    import bz_inputs as bi
    if w.get("R") is not None:
        R = w["R"]
        L = bi.L_from_R(R)
    else:
        L = w["L"]
        R = bi.R_from_L(L)
    return L, R


def _fhat(w, L):
    import bz_inputs as bi
    N = w["N"]
    if w["data"] == "bkw":
        return bi.bkw_fhat(N, L, bi.bkw_K(w["t0"]))
    if w["data"] == "c3":
        return bi.bigaussian_noise_c3(N, L)
    if w["data"] == "bkw2d":
        return bi.bkw2d_fhat_samples(N, L, bi.bkw2d_K(0.0))
    if w["data"] == "inhom":
        return bi.inhom_cells(N, L, w["nx"], w["Lx"])[0]      # one cell (the oracle's collide rate)
    return bi.two_maxwellians_c1(N, L)


def _flops_per_term(N, dim=3):
    """Algorithmic FP32 flops of one term (the per-unit count of the method's cost): two
    d-dimensional FFTs of n = N^d points at 5 n log2 n each, and 26 pointwise flops per mode
    (forming and applying the separable twiddle, 12; the product with h, 6; the alpha weight, 6;
    the accumulation, 2).  Split per chunked kernel as each one executes them."""
    n = N ** dim
    if dim == 2:
        return {"fused": 20 * n * math.log2(N) + 26 * n, "reduce": 2 * n}
    return {"plane_inv": 10 * n * math.log2(N) + 12 * n,
            "pencil": 10 * n * math.log2(N) + 6 * n,
            "plane_fwd": 10 * n * math.log2(N) + 6 * n,
            "reduce": 2 * n,
            "fused": 30 * n * math.log2(N) + 26 * n}


def _bytes_per_term(N, dim=3):
    """Algorithmic HBM bytes per term of each kernel (complex64 = 8 B per mode): the method
    must stream alpha_p once per term; fhat, h and the chunk scratch of the chunked pipeline
    are sized to stay in L2 and are not counted."""
    n = N ** dim
    return {"plane_inv": 0, "pencil": 0, "reduce": 0,
            "plane_fwd": 8 * n,          # alpha_p
            "fused": 8 * n}              # alpha_p; the field stays on chip


_PROFILES = {
    # kernel kind: (summary under profiles/, kernel sources the summary was taken from)
    "fused": ("fused_rk4_n32.md", ("bz_fused_kernel.cuh", "bz_fft.cuh", "bz_cluster.cuh")),
    "mixed": ("mixed_rk4_n32.md", ("bz_mixed.cu", "bz_fft.cuh", "bz_cluster.cuh")),
    "fused_real": ("fused_real_rk4_n32.md", ("bz_fused_kernel.cuh", "bz_fft.cuh", "bz_cluster.cuh")),
    "pair3": ("pair3_rk4_n32.md", ("bz_pair3.cu", "bz_fft.cuh", "bz_cluster.cuh")),
    "n64:pipeline": ("chunked_single_n64.md", ("bz_collide.cu", "bz_chunk64.cu", "bz_fft.cuh")),
}


def _sources_hash(files):
    import hashlib
    src = os.path.join(ROOT, "paper_2004_11239_gb300", "csrc")
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(src, f), "rb").read())
    return h.hexdigest()[:16]


def _profiled_traffic(key):
    """DRAM bytes per launch from the committed ncu summary of `key` (the kernel on its
    workload), if the kernel sources still match the fingerprint recorded with it."""
    if key not in _PROFILES:
        return None
    name, files = _PROFILES[key]
    prof = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(prof):
        return None
    vals = {}
    for line in open(prof):
        if ":" in line and line.startswith("    "):
            k, v = line.strip().split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_sources_sha256_16") != _sources_hash(files):
        return None
    return float(vals["traffic_bytes_per_launch"])


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _alu_peak(peaks):
    """FP32 FMA peak of the current device: SMs (queried) x 128 FP32 lanes x 2 flops x the
    measured maximum SM clock; returns (TFLOP/s, SM count, how it was derived)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = peaks.get("sm_max_mhz", 2070.0)
    return (sms * 128 * 2 * mhz * 1e6 / 1e12, sms,
            f"derived: {sms} SMs (device query) x 128 FP32 lanes x 2 x sm_max_mhz {mhz:.0f}")


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples every 200 ms during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(x: float) -> float:
    """Maximum of a per-rank float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, ms_local: float):
    """Whole-job units per second: all ranks' units over the slowest rank's time (replicas)."""
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    ms = max_over_ranks(ms_local)
    return units_per_rank * ws / (ms / 1e3), ms


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------------------
# The FP64 oracle on the host cores: one spawned process per core, each holding the oracle
# plan (F table) of one contiguous term range; a collide sends f to every process and adds
# their partial sums.  Used by the cpu_baseline leg, the reference arm and the measured error.
# ---------------------------------------------------------------------------------------

def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(conn, spec, p0, p1):
    """Serves one term range: ("plan",) builds the F table of [p0, p1); ("collide", f, real)
    returns (partial Q over the range, seconds); ("at", f, kidx, real) returns the partial Q at
    the modes kidx (F computed at those modes only); ("stop",) ends."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"                      # one core per process
    import numpy as np
    from oracle import ftable, kernels, spectral, spectral2d
    dim2 = spec.get("dim", 3) == 2
    kern = kernels.Kernel2D(spec["kernel2d"]) if dim2 else kernels.Kernel("family", spec["s"])
    plan = lite = None
    while True:
        msg = conn.recv()
        if msg[0] == "stop":
            break
        if msg[0] == "plan":
            t0 = time.perf_counter()
            if dim2:
                plan = spectral2d.OraclePlan2D(spec["N"], spec["L"], spec["R"], spec["gamma"], kern, spec["N_rho"],
                                               spec["M"])
            else:
                plan = spectral.OraclePlan(spec["N"], spec["L"], spec["R"], spec["gamma"], kern, spec["N_rho"],
                                           spec["M"], terms=np.arange(p0, p1))
            conn.send(time.perf_counter() - t0)
        elif msg[0] == "collide":
            f, real = msg[1], msg[2]
            t0 = time.perf_counter()
            if dim2:
                q = spectral2d.collide2d(plan, f, p0, p1)
            else:
                q = (spectral.collide_real if real else spectral.collide)(plan, f, p0, p1)
            conn.send((q, time.perf_counter() - t0))
        elif msg[0] == "at":
            f, kidx, real = msg[1], msg[2], msg[3]
            if lite is None:
                lite = spectral.OraclePlan(spec["N"], spec["L"], spec["R"], spec["gamma"], kern, spec["N_rho"],
                                           spec["M"], with_table=False)
            ks = spectral.signed(spec["N"])[kidx]
            n = p1 - p0
            F_at = ftable.fentries(spec["N"], spec["L"], np.repeat(ks, n, axis=0), np.tile(lite.r[p0:p1], len(ks)),
                                   np.tile(lite.q[p0:p1], (len(ks), 1)), kern).reshape(len(ks), n)
            g = spectral.real_band(f) if real else f
            conn.send(spectral.collide_at(lite, g, kidx, F_at, p0, p1))


class OracleCores:
    """The oracle spread over processes, one term range each (spawned: no fork after CUDA)."""

    def __init__(self, spec, ranges):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.ranges = [(a, b) for a, b in ranges if b > a]
        self.conns, self.procs = [], []
        for a, b in self.ranges:
            parent, child = ctx.Pipe()
            proc = ctx.Process(target=_oracle_worker, args=(child, spec, a, b), daemon=True)
            proc.start()
            self.conns.append(parent)
            self.procs.append(proc)

    @property
    def terms(self):
        return sum(b - a for a, b in self.ranges)

    def build(self):
        for c in self.conns:
            c.send(("plan",))
        return max(c.recv() for c in self.conns)

    def collide(self, f, real):
        """(sum of the partial Q over the ranges, wall seconds of the parallel region)."""
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(("collide", f, real))
        parts = [c.recv() for c in self.conns]
        return sum(q for q, _ in parts), time.perf_counter() - t0

    def at(self, f, kidx, real):
        for c in self.conns:
            c.send(("at", f, kidx, real))
        return sum(c.recv() for c in self.conns)

    def close(self):
        for c in self.conns:
            try:
                c.send(("stop",))
            except OSError:
                pass
        for p in self.procs:
            p.join(timeout=10)


def _split(p0, p1, parts):
    """Contiguous near-equal ranges covering [p0, p1)."""
    n = p1 - p0
    cuts = [p0 + (n * i) // parts for i in range(parts + 1)]
    return list(zip(cuts[:-1], cuts[1:]))


def _oracle_spec(w, L, R):
    spec = {"N": w["N"], "L": L, "R": R, "gamma": w["gamma"], "s": w["s"], "N_rho": w["N_rho"], "M": w["M"],
            "dim": w.get("dim", 3)}
    if spec["dim"] == 2:
        spec["kernel2d"] = {3: "b1", 4: "b2", 5: "b3", 6: "b4"}[w["kernel"]]
    return spec


def cpu_baseline_cores(w, L, R, f, real, target_s=15.0):
    """The FP64 oracle on every host core on a bounded sample: each process builds the F table
    of a few consecutive terms (a one-time plan cost, not timed) and runs the operator over them
    until about target_s of CPU work is done in all; evals/s = (terms per second over all
    processes) / P."""
    cores = _host_cores()
    P = w["N_rho"] * w["M"]
    per = max(1, min(P // cores, 2))
    starts = [int(x) for x in (P - per) * (0.5 + __import__("numpy").arange(cores)) / cores]
    oc = OracleCores(_oracle_spec(w, L, R), [(a, a + per) for a in starts])
    try:
        oc.build()
        _, t1 = oc.collide(f, real)                  # one pass: the rate estimate
        reps = max(1, int(target_s / cores / max(t1, 1e-3)))
        t0 = time.perf_counter()
        for _ in range(reps):
            oc.collide(f, real)
        wall = time.perf_counter() - t0
    finally:
        oc.close()
    rate = oc.terms * reps / wall                   # terms per second, all processes
    return {"value": rate / P, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{per} terms per process x {cores} processes (one per host core), {reps} passes of the "
                      f"operator over them ({oc.terms} of {P} terms of one N={w['N']} collide), terms per second "
                      f"/ P; the F-table build (a one-time plan cost) is excluded"}


def sampled_modes(q_gpu, n_top=64, n_rand=128, n_nyq=64, seed=12):
    """Modes at which the oracle checks a collide (array indices [S, 3]): the n_top largest
    |Qhat|, n_rand seeded uniform ones, and n_nyq seeded ones on the Nyquist planes (an index
    N/2 on some axis, where the real-data form and eq. realQ differ most)."""
    import numpy as np
    import bz_inputs as bi
    N = q_gpu.shape[0]
    top = np.argsort(np.abs(q_gpu).ravel())[::-1][:n_top]
    u = bi.SplitMix64(seed).uniform(n_rand + 3 * n_nyq)
    rnd = (u[:n_rand] * N ** 3).astype(np.int64)
    v = (u[n_rand:].reshape(n_nyq, 3) * N).astype(np.int64)
    v[np.arange(n_nyq), np.arange(n_nyq) % 3] = N // 2
    nyq = (v[:, 0] * N + v[:, 1]) * N + v[:, 2]
    flat = np.unique(np.concatenate([top, rnd, nyq]))
    return np.stack(np.unravel_index(flat, q_gpu.shape), axis=1)


def error_vs_oracle(w, L, R, f, q_gpu, p0=0, p1=None, real=False, also_realq=False):
    """Relative L-infinity error of a GPU collide (terms [p0, p1)) against the FP64 oracle at the
    sampled modes: max_s |Q_gpu(k_s) - Q_oracle(k_s)| / max_k |Q_gpu(k)|, the oracle spread over
    the host cores.  real: against the real-data reading; also_realq: also against eq. realQ on
    the unmodified input."""
    import numpy as np
    P = w["N_rho"] * w["M"]
    p1 = P if p1 is None else p1
    kidx = sampled_modes(q_gpu)
    t0 = time.perf_counter()
    oc = OracleCores(_oracle_spec(w, L, R), _split(p0, p1, min(_host_cores(), p1 - p0)))
    try:
        ref = oc.at(f, kidx, real)
        ref2 = oc.at(f, kidx, False) if (real and also_realq) else None
    finally:
        oc.close()
    norm = float(np.max(np.abs(q_gpu)))
    got = q_gpu[kidx[:, 0], kidx[:, 1], kidx[:, 2]]
    out = {"rel_linf": float(np.max(np.abs(got - ref)) / norm), "modes": int(len(kidx)), "terms": [p0, p1],
           "reference": "real-data reading (Hermitian, Nyquist-free part of f)" if real else "eq. realQ",
           "oracle_s": time.perf_counter() - t0, "cores": _host_cores()}
    if ref2 is not None:
        out["rel_linf_vs_eq_realQ"] = float(np.max(np.abs(got - ref2)) / norm)
    return out


def run_reference(args, w):
    """The FP64 oracle on the host cores, on this arm's workload, metric and unit: a step is
    the same unit as the GPU arm's (an RK4 step = 4 full collides through the oracle's RK4
    stage formula, or one full collide) when K + W of them fit in about three minutes, else a
    full collide's terms sampled evenly (extrapolated).  Rank 0 only."""
    import numpy as np
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import spectral
    L, R = _geometry(w)
    f = _fhat(w, L)
    real = args.data == "real" or (args.data == "auto" and _real_supported(w))
    cores = _host_cores()
    P = w["N_rho"] * w["M"]
    is_rk = w["dt"] is not None
    budget = 180.0
    # estimate from one term per core: F-table seconds per term and operator seconds per term
    starts = [a for a, _ in _split(0, P, cores)]
    probe = OracleCores(_oracle_spec(w, L, R), [(a, a + 1) for a in starts])
    try:
        tf = probe.build()
        _, tc = probe.collide(f, real)
    finally:
        probe.close()
    collide_s = tc * P / cores                       # wall of one full collide on every core
    steps = args.steps + args.warmup
    if is_rk and steps * 4 * collide_s + tf * P / cores < budget:
        mode, terms = "rk4", P
    elif steps * collide_s + tf * P / cores < budget:
        mode, terms = "collide", P
    else:
        mode = "sample"
        terms = max(cores, min(P, int(budget / steps / max(tc, 1e-6) * cores / 2)))
    ranges = _split(0, P, cores) if terms == P else [(a, a + max(1, terms // cores)) for a in starts]
    oc = OracleCores(_oracle_spec(w, L, R), ranges)
    try:
        oc.build()
        frac = P / oc.terms

        def rhs(g):
            q, _ = oc.collide(g, real)
            return q

        times = []
        fcur = f.copy()
        for i in range(steps):
            t0 = time.perf_counter()
            if mode == "rk4":
                fcur = spectral.rk4_steps(rhs, fcur, w["dt"], 1)
            else:
                rhs(fcur)
            dt_s = time.perf_counter() - t0
            if i >= args.warmup:
                times.append(dt_s)
    finally:
        oc.close()
    evals_per_step = 4 if mode == "rk4" else 1
    sec_per_step = statistics.median(times) * (frac if mode == "sample" else 1.0)
    value = evals_per_step / sec_per_step
    sample = {"rk4": f"full RK4 steps (4 full collides of all {P} terms each) on {cores} host cores",
              "collide": f"one full collide (all {P} terms) per step on {cores} host cores",
              "sample": f"{oc.terms} of {P} terms of one collide per step on {cores} host cores, "
                        f"extrapolated to all terms"}[mode]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(args, w, real),
            "collides_per_step": evals_per_step,
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": sample + "; the F-table build (a one-time plan cost) is excluded"},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _config(args, w, real):
    """The workload as both arms name it."""
    return {"workload": args.workload, "desc": w["desc"], "P": w["N_rho"] * w["M"],
            "data_form": "real" if real else "complex"}


def _real_supported(w):
    """The real-data form (BZ_DATA_REAL) applies to 3D plans with M even (fused pair kernels for
    N dividing 32, the chunked pipeline otherwise); the workloads' distribution functions are real."""
    return w.get("dim", 3) == 3 and w["M"] % 2 == 0


def _time_plan(args, w, bz, plan, f, q, st, barrier, clk=None):
    """W warm-up steps, then K steps between barriers and synchronisations (the throughput), then
    K more steps with the library's per-kernel CUDA events on (the roofline's kernel times; the
    event records add host work between launches, so they stay out of the throughput region).
    Returns (evals/s over all ranks, ms, per-kernel timings, launches per step, step)."""
    import torch
    is_rk = w["dt"] is not None
    evals_per_step = 4 if is_rk else 1

    def step():
        if is_rk:
            bz.bz_step_rk(plan, f, 0.0, w["dt"], 1, st)
        else:
            bz.bz_collide(plan, f, q, st)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches_per_step = bz.bz_plan_last_launches(plan)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if clk is not None:
        clk.__enter__()
    barrier()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    if clk is not None:
        clk.__exit__(None, None, None)
    ms = e0.elapsed_time(e1)
    value, ms = job_throughput(evals_per_step * args.steps, ms)
    bz.bz_plan_set_timing(plan, launches_per_step * args.steps + 16)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    kern = {name: bz.bz_plan_timing(plan, kind) for name, kind in bz.KERNEL_KINDS.items()}
    bz.bz_plan_set_timing(plan, 0)
    return value, ms, kern, launches_per_step, step


def _roofline(args, w, kern, peaks, src, profile_key):
    """Roofline of the dominant kernel: algorithmic flops and HBM bytes per term (the per-unit
    figures of the method, whatever form executes them) x terms per launch / mean launch time."""
    N, dim = w["N"], w.get("dim", 3)
    evals_per_step = 4 if w["dt"] is not None else 1
    dom = max(("plane_inv", "pencil", "plane_fwd", "reduce", "fused"), key=lambda k: kern[k][1])
    n_launch, ms_k = kern[dom]
    terms_per_launch = (w["N_rho"] * w["M"]) * evals_per_step * args.steps / max(n_launch, 1)
    if dom == "reduce" and kern["fused"][0] > 0:
        terms_per_launch = 0.0            # the partial-sum reduction is not a per-term kernel
    avg_s = ms_k / 1e3 / max(n_launch, 1)
    fl = _flops_per_term(N, dim).get(dom, 0.0) * terms_per_launch
    by = _bytes_per_term(N, dim).get(dom, 0.0) * terms_per_launch
    alu_peak, sms, alu_src = _alu_peak(peaks)
    alu = {"bound": "alu", "achieved": fl / avg_s / 1e12, "peak": alu_peak, "unit": "TFLOP/s"}
    hbm = {"bound": "hbm", "achieved": by / avg_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    for r in (alu, hbm):
        r["frac"] = r["achieved"] / r["peak"]
    roof = max((alu, hbm), key=lambda r: r["frac"])
    other = hbm if roof is alu else alu
    if profile_key == "n64":
        key = f"n64:{dom}"                 # the chunked kernels at N = 64, P = 4096
    elif args.workload == "rk4_n32" and dom == "fused":
        key = profile_key
    else:
        key = None
    roof.update({"kernel": dom, "traffic": _profiled_traffic(key),
                 "peak_source": f"{src}" if roof is hbm else alu_src, "sm_count": sms,
                 "launches": n_launch, "avg_launch_us": avg_s * 1e6,
                 "also": {k: other[k] for k in ("bound", "achieved", "peak", "unit", "frac")}})
    return roof


def run_sharded(args, w):
    """Under torchrun with N > 1 ranks, the single-collide workloads shard the terms (strong
    scaling): per step each rank evaluates its term range with bz_collide_terms and one NCCL
    all-reduce of the N^3 complex128 result completes Qhat on every rank; value = collides per
    second of the whole job (each collide counted once), max time over ranks."""
    import torch
    import torch.distributed as dist
    ws, rank, local = _dist()
    dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2004_11239_gb300 as bz
    from paper_2004_11239_gb300 import shard
    L, R = _geometry(w)
    real = args.data == "real" or (args.data == "auto" and _real_supported(w))
    plan = bz.bz_plan_create_ex(w["N"], L, R, w["gamma"], w["s"], w["N_rho"], w["M"],
                                data=bz.BZ_DATA_REAL if real else bz.BZ_DATA_COMPLEX)
    f_host = _fhat(w, L)
    f = torch.from_numpy(f_host).to("cuda")
    q = torch.empty_like(f)
    p0, p1 = bz.bz_partition_terms(plan.P, plan.data, ws, rank)

    def step():
        shard.collide_sharded(plan, f, q)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches = bz.bz_plan_last_launches(plan)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(local)
    clk.__enter__()
    dist.barrier()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    dist.barrier()
    clk.__exit__(None, None, None)
    ms = max_over_ranks(e0.elapsed_time(e1))
    value = args.steps / (ms / 1e3)
    # end to end: the input copied from pinned host memory to every rank, the result read back
    h_in = torch.from_numpy(f_host).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    dist.barrier()
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record()
    for _ in range(args.steps):
        f.copy_(h_in, non_blocking=True)
        step()
        h_out.copy_(q, non_blocking=True)
    e3.record()
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e2.elapsed_time(e3))
    nbytes = f.numel() * f.element_size()
    if rank == 0:
        cfg = _config(args, w, real)
        cfg.update({"terms_per_rank": [list(bz.bz_partition_terms(plan.P, plan.data, ws, r)) for r in range(ws)],
                    "exchange": "one NCCL all-reduce (sum) of the N^3 complex128 result per collide",
                    "l2": "inputs larger than L2: each rank streams its slice of the pair or alpha table"})
        print(json.dumps({"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                          "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                          "config": cfg, "clocks": clk.summary(), "gpu_launches": launches * args.steps,
                          "e2e": {"value": args.steps / (ms_e2e / 1e3), "unit": "evals/s",
                                  "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}}))
    plan.close()
    dist.destroy_process_group()
    return 0


def _pipeline_roofline(w, ms_per_collide, peaks, src, traffic_key=None):
    """Roofline of a whole collide on the chunked pipeline, whose kernels overlap on two streams:
    the method's algorithmic flops (the per-term count of `_flops_per_term`, every term) and
    the alpha-table bytes (8 N^3 per term) of one collide over the measured collide time,
    against the FP32 FMA peak and the measured HBM bandwidth; the larger fraction binds."""
    N, P = w["N"], w["N_rho"] * w["M"]
    s = ms_per_collide / 1e3
    alu_peak, sms, alu_src = _alu_peak(peaks)
    alu = {"bound": "alu", "achieved": _flops_per_term(N)["fused"] * P / s / 1e12, "peak": alu_peak,
           "unit": "TFLOP/s"}
    hbm = {"bound": "hbm", "achieved": _bytes_per_term(N)["fused"] * P / s / 1e9, "peak": peaks["hbm_gbs"],
           "unit": "GB/s"}
    for r in (alu, hbm):
        r["frac"] = r["achieved"] / r["peak"]
    roof, other = (alu, hbm) if alu["frac"] >= hbm["frac"] else (hbm, alu)
    roof.update({"kernel": "chunked pipeline (plane, pencil, plane, reduce on two streams)",
                 "traffic": _profiled_traffic(traffic_key) if traffic_key else None,
                 "peak_source": alu_src if roof is alu else src, "sm_count": sms,
                 "avg_launch_us": ms_per_collide * 1e3, "unit_of_work": f"one collide of {P} terms",
                 "also": {k: other[k] for k in ("bound", "achieved", "peak", "unit", "frac")}})
    return roof


def _bkw_trajectory(bz, plan, w, L, steps=500):
    """The BKW trajectory check: RK4 of the BKW solution from t0 for `steps` steps of dt on the GPU
    (complex128 state), against the exact BKW solution (Sec. 5.1, eq. BKW) at the final time:
    relative L-infinity error of the coefficients, max |f_gpu - f_exact| / max |f_exact|.
    This measures the method (quadrature, truncation) and the FP32 pipeline together."""
    import numpy as np
    import torch
    import bz_inputs as bi
    t0, dt = w["t0"], w["dt"]
    f = torch.from_numpy(bi.bkw_fhat(w["N"], L, bi.bkw_K(t0))).to("cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    t = bz.bz_step_rk(plan, f, t0, dt, steps)
    e1.record()
    torch.cuda.synchronize()
    exact = bi.bkw_fhat(w["N"], L, bi.bkw_K(t))
    got = f.cpu().numpy()
    start = bi.bkw_fhat(w["N"], L, bi.bkw_K(t0))
    return {"t0": t0, "t_end": t, "steps": steps, "dt": dt, "ms": e0.elapsed_time(e1),
            "rel_linf_vs_bkw": float(np.max(np.abs(got - exact)) / np.max(np.abs(exact))),
            "rel_change_of_f": float(np.max(np.abs(exact - start)) / np.max(np.abs(exact)))}


def run_ours(args, w):
    import numpy as np
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2004_11239_gb300 as bz

    L, R = _geometry(w)
    N = w["N"]
    dim = w.get("dim", 3)
    real = args.data == "real" or (args.data == "auto" and _real_supported(w))
    if real and not _real_supported(w):
        raise SystemExit("the real-data form needs a 3D plan with M even")
    data_form = bz.BZ_DATA_REAL if real else bz.BZ_DATA_COMPLEX

    def make_plan(form):
        return bz.bz_plan_create_ex(N, L, R, w["gamma"], w["s"], w["N_rho"], w["M"], h_precision=args.h_precision,
                                    kernel=w.get("kernel", 0), dim=dim, data=form, cluster=args.cluster,
                                    ctas_per_sm=args.ctas_per_sm if form == bz.BZ_DATA_REAL else 0)

    plan = make_plan(data_form)
    pipe = bz.bz_plan_pipeline(plan)
    pipe["h_precision"] = {0: "fp64", 1: "fp64", 2: "fp32"}[args.h_precision]
    f_host = _fhat(w, L)
    f = torch.from_numpy(f_host).to("cuda")
    q = torch.empty_like(f)
    st = torch.cuda.current_stream()
    is_rk = w["dt"] is not None
    evals_per_step = 4 if is_rk else 1

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    clk = ClockSampler(local)
    value, ms, kern, launches_per_step, step = _time_plan(args, w, bz, plan, f, q, st, barrier, clk)
    clocks = clk.summary()

    # end to end through the public API with host buffers (pinned), copies inside the region
    h_in = torch.from_numpy(f_host).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e2.record(st)
    for _ in range(args.steps):
        f.copy_(h_in, non_blocking=True)
        step()
        h_out.copy_(f if is_rk else q, non_blocking=True)
    e3.record(st)
    torch.cuda.synchronize()
    ms_e2e = e2.elapsed_time(e3)
    nbytes = f.numel() * f.element_size()
    e2e = {"value": evals_per_step * args.steps * ws / (ms_e2e / 1e3), "unit": "evals/s",
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    peaks, src = _peaks()
    kname = pipe.get("kernel", "k_fused")
    if pipe["pipeline"] == "chunked" and not is_rk:
        roof = _pipeline_roofline(w, ms / args.steps, peaks, src,
                                  "n64:pipeline" if (args.workload == "single_n64" and real) else None)
    else:
        roof = _roofline(args, w, kern, peaks, src, "pair3" if kname == "k_pair3" else ("fused_real" if real else "fused"))
    roof["kernel_name"] = kname
    if real:
        roof["executed"] = ("term pairs share every pair of 3D transforms: about half the counted FFT "
                            "flops and half the alpha bytes (plus a 3 N^2 Nyquist table per pair) are executed")

    # the other data form on the same workload (complex beside real, and the reverse where it applies)
    other = None
    if dim == 3 and (real or _real_supported(w)) and not args.no_other_form:
        po = make_plan(bz.BZ_DATA_COMPLEX if real else bz.BZ_DATA_REAL)
        fo, qo = torch.from_numpy(f_host).to("cuda"), torch.empty_like(f)
        qa = torch.empty_like(f)
        bz.bz_collide(plan, fo, qa, st)
        bz.bz_collide(po, fo, qo, st)
        torch.cuda.synchronize()
        a, b = qa.cpu().numpy(), qo.cpu().numpy()
        dev = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
        vo, mso, kerno, lo, _ = _time_plan(args, w, bz, po, fo, qo, st, barrier)
        other = {"data_form": "complex" if real else "real", "value": vo, "unit": "evals/s",
                 "ms_per_step": mso / args.steps, "gpu_launches": lo * args.steps,
                 "rel_linf_headline_vs_this": dev,
                 "roofline": _roofline(args, w, kerno, peaks, src, "fused" if real else "fused_real")}
        po.close()

    # the same workload with h formed in FP32 too: FP64 only in the weight tables, the RK state
    # and the moments
    pure = None
    if args.workload == "rk4_n32" and real and args.h_precision != 2 and not args.no_other_form:
        pp = bz.bz_plan_create_ex(N, L, R, w["gamma"], w["s"], w["N_rho"], w["M"], h_precision=2, data=data_form)
        fp, qp = torch.from_numpy(f_host).to("cuda"), torch.empty_like(f)
        vp, msp, kernp, lp, _ = _time_plan(args, w, bz, pp, fp, qp, st, barrier)
        bz.bz_collide(pp, torch.from_numpy(f_host).to("cuda"), qp, st)
        torch.cuda.synchronize()
        pure = {"h_precision": "fp32", "value": vp, "unit": "evals/s", "ms_per_step": msp / args.steps,
                "kernel": bz.bz_plan_pipeline(pp)["kernel"], "gpu_launches": lp * args.steps}
        if rank == 0 and not args.no_cpu_baseline:
            pure["parity"] = error_vs_oracle(w, L, R, f_host, qp.cpu().numpy().astype(np.complex128), real=True,
                                             also_realq=True)
        pp.close()

    mixed = None
    if N == 32 and dim == 3 and not args.no_mixed:
        pc = plan if not real else make_plan(bz.BZ_DATA_COMPLEX)
        mixed = _measure_mixed(args, w, bz, pc, f_host, L, R, st, peaks, src, barrier)
        if pc is not plan:
            pc.close()

    # parity of one headline collide against the FP64 oracle (host cores), after the timed regions
    parity = None
    if rank == 0 and not args.no_cpu_baseline and dim == 3:
        f0 = torch.from_numpy(f_host).to("cuda")
        bz.bz_collide(plan, f0, q, st)
        torch.cuda.synchronize()
        parity = error_vs_oracle(w, L, R, f_host, q.cpu().numpy().astype(np.complex128), real=real,
                                 also_realq=real)
        parity["collide"] = "one full collide of the workload's input through bz_collide"

    # the 500-step BKW trajectory (t = 6.5 -> 11.5) against the exact solution, s = 1/2 and 1/4
    trajectory = None
    if args.workload == "rk4_n32" and not args.no_trajectory:
        trajectory = {"desc": "RK4 of the BKW solution from t=6.5 to t=11.5 (500 steps of 0.01), N=32, "
                              "N_rho=M=32, gamma=0, against the exact solution (eq. BKW) at t=11.5",
                      "s=0.5": _bkw_trajectory(bz, plan, w, L)}
        p25 = bz.bz_plan_create_ex(N, L, R, w["gamma"], 0.25, w["N_rho"], w["M"], data=data_form)
        trajectory["s=0.25"] = _bkw_trajectory(bz, p25, w, L)
        p25.close()

    n64 = None
    if args.workload == "rk4_n32" and not args.no_n64:
        n64 = _measure_n64(args, bz, peaks, src, barrier, rank == 0 and not args.no_cpu_baseline)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_cores(w, L, R, f_host, real)

    streamed = plan.alpha_bytes - (plan.P * N ** 3 * 8 if real else 0)
    form_desc = ("real: f is real, fhat's Hermitian part with the Nyquist planes (index -N/2) dropped "
                 "(BZ_DATA_REAL; `parity` gives its measured distance from eq. realQ on this input)" if real else
                 "complex: eq. realQ on fhat as given (BZ_DATA_COMPLEX)")
    config = _config(args, w, real)
    config.update({"data_form_desc": form_desc, "pipeline": pipe, "collides_per_step": evals_per_step,
                   "l2": "inputs larger than L2: the %s of %d MB streams every collide"
                         % ("pair table" if real else "alpha table", streamed >> 20)})
    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config,
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "roofline": roof, "kernels_ms": {k: v[1] for k, v in kern.items()},
            "parity": parity, "cpu_baseline": cpu}
    if trajectory is not None:
        line["trajectory"] = trajectory
    if pure is not None:
        line["fp32_h"] = pure
    if n64 is not None:
        line["n64"] = n64
    if other is not None:
        line["other_form"] = other
    if mixed is not None:
        line["mixed"] = mixed
    if rank == 0:
        print(json.dumps(line))
    plan.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


N64 = dict(N=64, N_rho=64, M=64, gamma=-1.0, s=0.5, R=None, L=10.0, dt=None, data="c3",
           desc="single collide, N=64, N_rho=64, M=64 (P=4096), gamma=-1, s=0.5, L=10, bi-Gaussian "
                "(T=2, 0.5, 0.5) plus 1% seeded noise; real-data form on the chunked pipeline")


def _measure_n64(args, bz, peaks, src, barrier, with_parity):
    """The single-instance heavy collide (N = 64, P = 4096, gamma = -1): evals/s over K collides,
    the dominant chunked kernel's roofline (per-kernel CUDA events over K more collides), and the
    relative L-infinity error against the FP64 oracle on one full collide at sampled modes."""
    import numpy as np
    import torch
    w = N64
    L, R = _geometry(w)
    t0 = time.perf_counter()
    plan = bz.bz_plan_create_ex(64, L, R, w["gamma"], w["s"], w["N_rho"], w["M"], data=bz.BZ_DATA_REAL)
    plan_s = time.perf_counter() - t0
    f_host = _fhat(w, L)
    f = torch.from_numpy(f_host).to("cuda")
    q = torch.empty_like(f)
    st = torch.cuda.current_stream()
    a = argparse.Namespace(**vars(args))
    a.steps = max(5, min(args.steps, 50))
    value, ms, kern, launches, _ = _time_plan(a, w, bz, plan, f, q, st, barrier)
    roof = _pipeline_roofline(w, ms / a.steps, peaks, src, "n64:pipeline")
    out = {"desc": w["desc"], "value": value, "unit": "evals/s", "steps": a.steps, "ms_per_collide": ms / a.steps,
           "gpu_launches": launches * a.steps, "plan_create_s": plan_s, "roofline": roof,
           "kernels_ms": {k: v[1] / a.steps for k, v in kern.items()}, "pipeline": bz.bz_plan_pipeline(plan),
           "l2": "inputs larger than L2: the 4.3 GB pair table streams every collide"}
    if with_parity:
        bz.bz_collide(plan, f, q, st)
        torch.cuda.synchronize()
        out["parity"] = error_vs_oracle(w, L, R, f_host, q.cpu().numpy().astype(np.complex128), real=True)
        out["parity"]["collide"] = "one full collide (all 4096 terms) through bz_collide"
    plan.close()
    return out


def _tc_flops_per_term(N):
    """Tensor-core flops of one term in the split-BF16 form: six one-axis DFTs, each N^2 lines x
    2N real outputs x 3 (split products) x 2N real inputs, 2 flops per multiply-add."""
    return 6 * 2 * N ** 2 * (2 * N) * 3 * (2 * N)


def _measure_mixed(args, w, bz, plan32, f_host, L, R, st, peaks, src, barrier):
    """The same workload on the split-BF16 tensor-core form (BZ_PREC_BF16X3): throughput, the
    deviation from the FP32 form on one collide of the input, and the dominant kernel's
    tensor-pipe roofline."""
    import numpy as np
    import torch
    N = w["N"]
    pm = bz.bz_plan_create_ex(N, L, R, w["gamma"], w["s"], w["N_rho"], w["M"], precision=bz.BZ_PREC_BF16X3)
    f = torch.from_numpy(f_host).to("cuda")
    q32, qm = torch.empty_like(f), torch.empty_like(f)
    bz.bz_collide(plan32, f, q32, st)
    bz.bz_collide(pm, f, qm, st)
    torch.cuda.synchronize()
    a, b = qm.cpu().numpy(), q32.cpu().numpy()
    dev = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    is_rk = w["dt"] is not None
    evals_per_step = 4 if is_rk else 1

    def step():
        if is_rk:
            bz.bz_step_rk(pm, f, 0.0, w["dt"], 1, st)
        else:
            bz.bz_collide(pm, f, qm, st)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches_per_step = bz.bz_plan_last_launches(pm)
    bz.bz_plan_set_timing(pm, launches_per_step * args.steps + 16)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    n_launch, ms_k = bz.bz_plan_timing(pm, bz.KERNEL_KINDS["fused"])
    bz.bz_plan_set_timing(pm, 0)
    value, ms = job_throughput(evals_per_step * args.steps, ms)
    errors = bz.bz_plan_device_errors(pm)
    traj = _bkw_trajectory(bz, pm, w, L) if (is_rk and not args.no_trajectory) else None
    terms_per_launch = (w["N_rho"] * w["M"]) * evals_per_step * args.steps / max(n_launch, 1)
    avg_s = ms_k / 1e3 / max(n_launch, 1)
    tc = _tc_flops_per_term(N) * terms_per_launch / avg_s / 1e12
    tc_peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
    fft = _flops_per_term(N)["fused"] * terms_per_launch / avg_s / 1e12
    pm.close()
    return {"precision": "bf16x3", "value": value, "unit": "evals/s", "ms_per_step": ms / args.steps,
            "rel_linf_vs_fp32_form": dev, "device_errors": errors, "trajectory_s=0.5": traj,
            "gpu_launches": launches_per_step * args.steps,
            "roofline": {"bound": "tensor", "kernel": "k_mixed", "achieved": tc, "peak": tc_peak,
                         "unit": "TFLOP/s", "frac": tc / tc_peak,
                         "traffic": _profiled_traffic("mixed" if args.workload == "rk4_n32" else None), "launches": n_launch,
                         "avg_launch_us": avg_s * 1e6,
                         "peak_source": f"{src} bf16 (sustained)" if "bf16_tflops_sustained" in peaks else src,
                         "work": "split-BF16 DFT-GEMM flops: 6 x 2 N^2 x 2N x 3 x 2N per term",
                         "fft_equivalent_tflops": fft}}


def run_batch(args, w):
    """The batched workload: 4096 independent instances in six (N, s) groups, one RK4 step each."""
    import numpy as np
    import torch
    import bz_inputs as bi
    import paper_2004_11239_gb300 as bz
    torch.cuda.set_device(0)
    L = w["L"]
    R = bi.R_from_L(L)
    u = bi.SplitMix64(2024).uniform(2 * 4096)
    svals, gvals = [0.25, 0.5, 0.75], [0.0, -1.0]
    groups = {}
    for i in range(4096):
        N = 16 if i < 3072 else 32
        s_ = svals[int(u[2 * i] * 3)]
        g_ = gvals[int(u[2 * i + 1] * 2)]
        groups.setdefault((N, s_), []).append((i, g_))
    runs = []
    form = bz.BZ_DATA_COMPLEX if args.data == "complex" else bz.BZ_DATA_REAL    # M = 32 and N | 32: real applies
    for (N, s_), members in sorted(groups.items()):
        plan = bz.bz_plan_create_ex(N, L, R, 0.0, s_, N, w["M"], data=form)
        batch = bz.bz_batch_create(plan, len(members), 0)
        for slot, (i, g_) in enumerate(members):
            if g_ != 0.0:
                bz.bz_batch_set_gamma(batch, slot, g_)
        f = np.stack([bi.random_mixture(N, L, seed=i) for i, _ in members]).astype(np.complex64)
        fd = torch.from_numpy(f).cuda()
        runs.append((N, s_, plan, batch, fd, list(range(len(members))), torch.cuda.Stream()))
    def step():
        for N, s_, plan, batch, fd, slots, st in runs:
            bz.bz_batch_step_rk(batch, slots, fd, w["dt"], 1, st)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        e0.record()
        for *_, st in runs:
            st.wait_event(e0)
        for _ in range(args.steps):
            step()
        for *_, st in runs:
            torch.cuda.current_stream().wait_stream(st)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    wall = time.perf_counter() - t0
    evals = 4 * 4096 * args.steps
    launches = sum(bz.bz_batch_last_launches(r[3]) for r in runs) * args.steps
    # whole-step roofline: algorithmic FP32 flops of every term of every instance (the batch
    # shares each group's alpha table, so the step is bound by the CUDA cores, not by HBM)
    flops = sum(4 * len(r[5]) * r[2].P * _flops_per_term(r[0])["fused"] for r in runs) * args.steps
    peaks, _ = _peaks()
    alu_peak, sms, alu_src = _alu_peak(peaks)
    achieved = flops / (ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
            "kernel": "whole step (k_fused dominant)", "traffic": None,
            "peak_source": alu_src, "sm_count": sms,
            "work": "30 N^3 log2 N + 26 N^3 flops per term, 4 collides per RK4 step"}
    line = {"metric": METRIC, "value": evals / (ms / 1e3), "unit": "evals/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": args.workload, "desc": w["desc"],
                                            "data_form": "complex" if form == bz.BZ_DATA_COMPLEX else "real",
                                            "groups": {f"N={k[0]},s={k[1]}": len(v) for k, v in sorted(groups.items())},
                                            "terms_per_item": {f"N={r[0]},s={r[1]}": r[3].terms_per_item for r in runs}},
            "clocks": clk.summary(), "gpu_launches": launches, "wall_s": wall, "roofline": roof}
    print(json.dumps(line))
    return 0


def run_inhom(args, w):
    """The inhomogeneous workload: Strang steps over nx cells (free streaming and the batched RK4
    collision of every cell); evals = 4 collides per cell per step."""
    import numpy as np
    import torch
    import bz_inputs as bi
    import paper_2004_11239_gb300 as bz
    torch.cuda.set_device(0)
    L, R = _geometry(w)
    N, nx, Lx = w["N"], w["nx"], w["Lx"]
    form = bz.BZ_DATA_COMPLEX if args.data == "complex" else bz.BZ_DATA_REAL
    plan = bz.bz_plan_create_ex(N, L, R, w["gamma"], w["s"], w["N_rho"], w["M"], data=form)
    batch = bz.bz_batch_create(plan, nx, 0)
    f_host = bi.inhom_cells(N, L, nx, Lx)
    fd = torch.from_numpy(f_host).cuda()
    st = torch.cuda.current_stream()

    def step():
        bz.bz_inhom_step(batch, nx, Lx, fd, w["dt"], 1, st)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches = bz.bz_batch_last_launches(batch)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(args.steps):
            step()
        e1.record(st)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # the free-streaming share: the same number of transport calls alone (two per step)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(st)
    for _ in range(args.steps):
        bz.bz_transport_x(N, L, nx, Lx, fd, 0.5 * w["dt"], st)
        bz.bz_transport_x(N, L, nx, Lx, fd, 0.5 * w["dt"], st)
    e3.record(st)
    torch.cuda.synchronize()
    ms_tr = e2.elapsed_time(e3)
    # end to end: host cells copied in and out around every step
    h_in = torch.from_numpy(f_host).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e4.record(st)
    for _ in range(args.steps):
        fd.copy_(h_in, non_blocking=True)
        step()
        h_out.copy_(fd, non_blocking=True)
    e5.record(st)
    torch.cuda.synchronize()
    ms_e2e = e4.elapsed_time(e5)
    evals = 4 * nx * args.steps
    nbytes = fd.numel() * fd.element_size()
    flops = 4 * nx * plan.P * _flops_per_term(N)["fused"] * args.steps
    peaks, _ = _peaks()
    alu_peak, sms, alu_src = _alu_peak(peaks)
    achieved = flops / (ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
            "kernel": "whole step (k_fused dominant)", "traffic": None,
            "peak_source": alu_src, "sm_count": sms,
            "work": "30 N^3 log2 N + 26 N^3 flops per term, 4 collides per cell per step"}
    line = {"metric": METRIC, "value": evals / (ms / 1e3), "unit": "evals/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": args.workload, "desc": w["desc"], "cells": nx,
                                            "data_form": "complex" if form == bz.BZ_DATA_COMPLEX else "real",
                                            "P": plan.P, "transport_ms_per_step": ms_tr / args.steps,
                                            "transport_share": ms_tr / ms},
            "clocks": clk.summary(), "gpu_launches": launches * args.steps, "roofline": roof,
            "e2e": {"value": evals / (ms_e2e / 1e3), "unit": "evals/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes}}
    print(json.dumps(line))
    batch.close()
    plan.close()
    return 0


def _serve_trace(n_req, seed=77):
    """The serving workload's requests: N from {16, 24, 32, 48, 64}, N_rho = N, M from {12, 32},
    gamma from {0, -1, -2}, s from {0.25, 0.5}, seeded two-Maxwellian initial data."""
    import bz_inputs as bi
    u = bi.SplitMix64(seed).uniform(4 * n_req)
    Ns, Ms, gs, ss = [16, 24, 32, 48, 64], [12, 32], [0.0, -1.0, -2.0], [0.25, 0.5]
    return [dict(N=Ns[int(u[4 * i] * 5)], M=Ms[int(u[4 * i + 1] * 2)], gamma=gs[int(u[4 * i + 2] * 3)],
                 s=ss[int(u[4 * i + 3] * 2)], seed=1000 + i) for i in range(n_req)]


def run_serve(args, w):
    """A seeded Poisson trace through bz_submit / bz_poll: latency percentiles and throughput, for
    the FP32 server (real-data form where M is even) and the mixed-precision one (split-BF16 at
    N = 32, complex data; FP32 elsewhere).  Plans are warmed before each trace."""
    import numpy as np
    import torch
    import bz_inputs as bi
    import paper_2004_11239_gb300 as bz
    torch.cuda.set_device(0)
    L = w["L"]
    R = bi.R_from_L(L)
    n_req, rate = args.serve_requests, 200.0
    trace = _serve_trace(n_req)
    f0 = {r["seed"]: bi.random_mixture(r["N"], L, seed=r["seed"]) for r in trace}
    t_end = w["t_end"]
    server = bz.bz_server_create(200 << 30, max_batch=32, terms_per_item=32)

    def form(r, mixed):
        if mixed and r["N"] == 32:
            return bz.BZ_DATA_COMPLEX, bz.BZ_PREC_BF16X3
        return bz.BZ_DATA_REAL, bz.BZ_PREC_FP32          # M in {12, 32}: the real-data form applies

    def submit(r, t_end_, mixed):
        data, prec = form(r, mixed)
        return bz.bz_submit(server, f0[r["seed"]], r["N"], L, R, r["gamma"], r["s"], r["N"], r["M"], 0.0, t_end_,
                            w["dt"], data=data, precision=prec)

    def wait(tickets):
        out = {}
        while len(out) < len(tickets):
            for t, N in tickets:
                if t not in out:
                    res = bz.bz_poll(server, t, N)
                    if res is not None:
                        out[t] = res
            time.sleep(0.0005)
        return out

    def key(r, mixed):
        data, prec = form(r, mixed)                      # every group is a batch: gamma per slot
        return (r["N"], r["M"], r["s"], data, prec)

    passes = []
    for mixed in (False, True):
        keys = {}
        for r in trace:
            keys.setdefault(key(r, mixed), r)
        tw = time.perf_counter()
        wait([(submit(r, w["dt"], mixed), r["N"]) for r in keys.values()])     # plans, batches, graphs
        warm_s = time.perf_counter() - tw
        arr = bi.poisson_arrivals(n_req, rate, seed=78)
        t0 = time.perf_counter()
        tickets = []
        with ClockSampler(0) as clk:
            for r, ta in zip(trace, arr):
                delay = t0 + ta - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets.append((submit(r, t_end, mixed), r["N"]))
            res = wait(tickets)
        wall = time.perf_counter() - t0
        lat = np.array([res[t][0].latency_s for t, _ in tickets])
        que = np.array([res[t][0].queue_s for t, _ in tickets])
        steps = sum(res[t][0].steps for t, _ in tickets)
        by_n = {}
        for (t, N) in tickets:
            by_n.setdefault(N, []).append(res[t][0].latency_s)
        failed = {}
        for (t, N), r in zip(tickets, trace):
            st = res[t][0].status
            if st != 0:
                k = f"N={N},M={r['M']},gamma={r['gamma']},s={r['s']}"
                failed.setdefault(k, {}).setdefault(str(st), 0)
                failed[k][str(st)] += 1
        passes.append({"failed": failed,
                       "precision": "bf16x3 at N=32, fp32 elsewhere" if mixed else "fp32",
                       "requests_per_s": n_req / wall, "q_evals_per_s": 4 * steps / wall, "wall_s": wall,
                       "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                       "queue_p50_s": float(np.percentile(que, 50)), "queue_p99_s": float(np.percentile(que, 99)),
                       "latency_p50_by_N_s": {str(k): float(np.percentile(v, 50)) for k, v in sorted(by_n.items())},
                       "all_ok": all(res[t][0].status == 0 for t, _ in tickets), "plans": len(keys),
                       "warm_s": warm_s, "clocks": clk.summary()})
        if args.no_mixed:
            break
    sweep = []
    if args.rates:
        # a rate sweep on the first requests of the trace (FP32): p50 / p99 latency per rate
        sub = trace[:args.sweep_requests]
        for rt in [float(x) for x in args.rates.split(",")]:
            arr = bi.poisson_arrivals(len(sub), rt, seed=79)
            t0 = time.perf_counter()
            tickets = []
            for r, ta in zip(sub, arr):
                delay = t0 + ta - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets.append((submit(r, t_end, False), r["N"]))
            res = wait(tickets)
            wall = time.perf_counter() - t0
            lat = np.array([res[t][0].latency_s for t, _ in tickets])
            sweep.append({"rate": rt, "requests": len(sub), "requests_per_s": len(sub) / wall,
                          "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                          "all_ok": all(res[t][0].status == 0 for t, _ in tickets)})
    server.close()
    head = passes[0]
    line = {"metric": "served requests/s", "value": head["requests_per_s"], "unit": "requests/s", "n_gpus": 1,
            "steps": n_req, "warmup": head["plans"], "ms_per_step": 1e3 * head["wall_s"] / n_req,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"] % n_req, "rate": rate},
            "latency_s": {"p50": head["latency_p50_s"], "p99": head["latency_p99_s"]},
            "queue_s": {"p50": head["queue_p50_s"], "p99": head["queue_p99_s"]},
            "q_evals_per_s": head["q_evals_per_s"], "passes": passes}
    if sweep:
        line["rate_sweep"] = sweep
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rk4_n32", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-rho", type=int, default=0,
                    help="override the workload's radial points (a smaller case of the same kernels, for profiling)")
    ap.add_argument("--sphere-m", type=int, default=0, help="override the workload's sphere points")
    ap.add_argument("--no-other-form", action="store_true",
                    help="skip timing the other data form (complex beside real) on the same workload")
    ap.add_argument("--no-trajectory", action="store_true",
                    help="skip the 500-step BKW trajectory check of the default workload")
    ap.add_argument("--no-n64", action="store_true",
                    help="skip the N = 64 single-collide block measured beside the default workload")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the split-BF16 tensor-core form (measured beside the FP32 form at N = 32)")
    ap.add_argument("--serve-requests", type=int, default=256, help="serve workload: requests in the trace")
    ap.add_argument("--rates", default=None,
                    help="serve workload: comma-separated arrival rates (req/s) of a sweep after the trace")
    ap.add_argument("--sweep-requests", type=int, default=64, help="serve workload: requests per rate of the sweep")
    ap.add_argument("--data", default="auto", choices=["auto", "real", "complex"],
                    help="data form of the headline plan: auto = real where the plan supports it "
                         "(3D, N in {8, 16, 32}, M even; the workloads' f are real), else complex")
    ap.add_argument("--cluster", type=int, default=0,
                    help="CTAs per cluster of the fused kernel (0: timed at plan creation, fastest kept)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, choices=[0, 2, 3],
                    help="real-data form at N = 32: 2 runs k_fused, 3 k_pair3, 0 times both at plan creation")
    ap.add_argument("--h-precision", type=int, default=0, choices=[0, 1, 2],
                    help="h = IFFT(fhat) precision on the fused path: 0 auto (FP64), 1 FP64, 2 FP32")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.n_rho > 0:
        w["N_rho"] = args.n_rho
        w["desc"] += f" [N_rho overridden: {args.n_rho}]"
    if args.sphere_m > 0:
        w["M"] = args.sphere_m
        w["desc"] += f" [M overridden: {args.sphere_m}]"
    if args.impl == "reference" and args.workload in ("batch_4096", "serve"):
        # the oracle computes one collide at a time: its rate on one instance is the reference
        ws, rank, _ = _dist()
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the FP64 oracle has no batched or served "
                              "form; its per-collide rate is the reference of --workload rk4_n32"}))
        return 0
    if args.workload == "batch_4096":
        return run_batch(args, w)
    if args.workload == "serve":
        return run_serve(args, w)
    if args.impl == "reference":
        return run_reference(args, w)
    if args.workload == "inhom_n16":
        return run_inhom(args, w)
    if _dist()[0] > 1 and w["dt"] is None and w.get("dim", 3) == 3:
        return run_sharded(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
