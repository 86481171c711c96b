"""The multi-GPU bench path is replicas only (one independent solve per rank,
no collective in the solver): its bookkeeping, the max over ranks of the timed
region and the whole-job value, runs here on two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = 1000.0 + 250.0 * rank            # rank 1 is the slow one
    m = bench.reduce_max(my_ms, dist, "cpu")
    q.put((rank, m, bench.whole_job_value(world, 4, m)))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in out:
        assert m == 1250.0
        assert v == pytest.approx(2 * 4 / 1.25)


def test_single_process_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.whole_job_value(1, 5, 2000.0) == pytest.approx(2.5)
