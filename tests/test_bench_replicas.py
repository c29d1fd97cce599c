"""The replica (N > 1) logic of bench.py on the CPU: two gloo ranks, the barrier, the
max-over-ranks timing and the whole-job throughput.  No GPU and no data-path collective."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    ms = bench.allreduce_max(1.5 + rank, world)           # rank 1 is the slow one
    out[rank] = (ms, bench.replica_throughput(4e9, ms, world))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5
    # 2 ranks x 4 GB in 2.5 ms
    assert abs(res[0][1] - 2 * 4e9 / 2.5e-3 / 1e9) < 1e-6


def test_single_rank_is_identity():
    import bench
    assert bench.allreduce_max(3.25, 1) == 3.25
    assert bench.replica_throughput(1e9, 1.0, 1) == pytest.approx(1000.0)
