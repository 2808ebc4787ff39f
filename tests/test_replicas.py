"""The multi-GPU path is replicas only (the block-tridiagonal chain and the contact solve couple
every node, so one instance does not shard): each rank solves its own sweep, and the job's
throughput is all ranks' solves over the slowest rank's time.  This checks that aggregation with
two gloo ranks on the CPU (rendezvous on 127.0.0.1)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r: 60 solves per step, 3 steps, device time 500 + 100 r ms, end-to-end 0.6 + 0.2 r s
    out = bench.replica_totals(500.0 + 100.0 * rank, 0.6 + 0.2 * rank, 180, world, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_replica_totals_take_the_slowest_rank_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        t_max, e2e_max, value, e2e_value = res[r]
        assert t_max == 600.0 and e2e_max == pytest.approx(0.8)
        assert value == pytest.approx(360 / 0.6) and e2e_value == pytest.approx(360 / 0.8)


def test_replica_totals_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_totals(500.0, 0.5, 180, 1) == (500.0, 0.5, 360.0, 360.0)
