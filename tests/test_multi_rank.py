"""Host-side logic of the N > 1 benchmark (independent replicas, max over ranks),
run as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]               # rank 1 is the slow replica
    ms_max = bench.reduce_max(ms, dist)
    val = bench.replica_value(world, per_cycle=1000.0, steps=4, ms_max=ms_max)
    dist.barrier()
    q.put((rank, ms_max, val))
    dist.destroy_process_group()


def test_two_rank_max_and_replica_value():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, val in out:
        assert ms_max == 150.0
        assert abs(val - 2 * 1000.0 * 4 / 0.150) < 1e-6
