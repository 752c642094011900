"""The bench's multi-rank aggregation (replicas, max over ranks) on two gloo ranks (CPU)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (r + 1) * 100 ms for 40 units
    value, ms = bench.job_throughput(40.0, 100.0 * (rank + 1))
    out[rank] = (value, ms, bench.max_over_ranks(float(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_uses_all_units_over_the_slowest_rank():
    mp = torch.multiprocessing.get_context("spawn")
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        value, ms, mx = out[r]
        assert ms == 200.0                     # the slowest rank's time on every rank
        assert abs(value - 80.0 / 0.2) < 1e-9  # 2 x 40 units in 0.2 s
        assert mx == 1.0


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    value, ms = bench.job_throughput(10.0, 500.0)
    assert ms == 500.0 and value == 20.0
