"""Term sharding of the collide (the multi-GPU form of eq. realQ, Sec. 4), on the CPU:
the host partition from the C ABI, and the partition-and-reduce step on two gloo ranks with the
FP64 oracle's partial sums standing in for each rank's GPU result."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bz():
    import __graft_entry__
    __graft_entry__._libbuild().build()
    import paper_2004_11239_gb300 as m
    return m


@pytest.mark.parametrize("P,data,world", [(1024, 0, 1), (1024, 0, 3), (4096, 1, 8), (24, 1, 5),
                                          (6, 0, 8), (10, 1, 7)])
def test_partition_covers_every_term_once(bz, P, data, world):
    ranges = [bz.bz_partition_terms(P, data, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == P
    assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    sizes = [b - a for a, b in ranges]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= (2 if data else 1)
    if data == 1:                                   # term pairs stay whole
        assert all(a % 2 == 0 and b % 2 == 0 for a, b in ranges)


def test_partition_rejects_bad_arguments(bz):
    for args in ((10, 0, 0, 0), (10, 0, 2, 2), (10, 0, 2, -1), (11, 1, 2, 0), (-1, 0, 1, 0), (10, 5, 1, 0)):
        with pytest.raises(bz.BzError) as e:
            bz.bz_partition_terms(*args)
        assert e.value.code == 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, real, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bz_inputs as bi
    from oracle import kernels, spectral
    from paper_2004_11239_gb300 import shard
    L = 6.0
    plan = spectral.OraclePlan(8, L, bi.R_from_L(L), -1.0, kernels.Kernel("family", 0.5), 3, 12)
    f = bi.random_mixture(8, L, seed=21, box=1.5)
    fn = spectral.collide_real if real else spectral.collide

    def partial(p0, p1):
        out[("range", rank)] = (p0, p1)
        return torch.from_numpy(fn(plan, f, p0, p1))

    q = shard.sharded_sum(plan.P, 1 if real else 0, world, rank, partial,
                          lambda t: dist.all_reduce(t, op=dist.ReduceOp.SUM))
    out[("q", rank)] = q.numpy()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("real", [False, True])
def test_two_gloo_ranks_reduce_to_the_full_collide(real):
    import bz_inputs as bi
    from oracle import kernels, spectral
    mp = torch.multiprocessing.get_context("spawn")
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, real, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    L = 6.0
    plan = spectral.OraclePlan(8, L, bi.R_from_L(L), -1.0, kernels.Kernel("family", 0.5), 3, 12)
    f = bi.random_mixture(8, L, seed=21, box=1.5)
    full = (spectral.collide_real if real else spectral.collide)(plan, f)
    r0, r1 = out[("range", 0)], out[("range", 1)]
    assert r0[0] == 0 and r0[1] == r1[0] and r1[1] == plan.P and 0 < r0[1] < plan.P
    for r in range(2):
        assert np.max(np.abs(out[("q", r)] - full)) < 1e-13 * np.max(np.abs(full))
