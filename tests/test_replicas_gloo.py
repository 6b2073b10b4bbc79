"""The N > 1 path of bench.py: every rank integrates an independent replica
and the whole-job value is the simulated time of all ranks over the slowest
rank's time.  Checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def rmax(x):
        v = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(v, op=dist.ReduceOp.MAX)
        return float(v.item())

    def rsum(x):
        v = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(v, op=dist.ReduceOp.SUM)
        return float(v.item())

    # rank r simulated 0.2 ns in 1 + r seconds
    value, t_max = bench.aggregate(0.2, 1.0 + rank, world, rmax, rsum)
    out.put((rank, value, t_max, bench.dist_env()))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_as_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t_max, env in res:
        assert t_max == pytest.approx(2.0)
        assert value == pytest.approx(0.4 / 2.0)
        assert env[0] == 2 and env[1] == rank
