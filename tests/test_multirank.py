"""Multi-process host logic of the benchmark (replicas, max over ranks) on CPU with the
gloo backend and two ranks: the whole-job value uses the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]  # rank 1 is the slow one
    t = torch.tensor([local_ms])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    value = bench.aggregate(world, 1000, 10, [float(t.item())])
    out[rank] = value
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    expect = 2 * 1000 * 10 / 0.25 / 1e9
    assert abs(out[0] - expect) < 1e-18 and abs(out[1] - expect) < 1e-18
