"""N > 1 replica logic of bench.py on CPU: two gloo ranks time different amounts of work; both
see the same job time (the maximum) and the whole-job throughput counts both ranks."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2112_14681_b300 import replicas
    r, lr, w = replicas.world()
    assert (r, lr, w) == (rank, rank, world)
    replicas.barrier(dist)
    seconds = 1.0 + rank  # rank 1 is slower
    value, tmax = replicas.aggregate_throughput(dist, 10, seconds)
    out[rank] = (value, tmax)
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_total_throughput():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        value, tmax = out[r]
        assert tmax == 2.0 and value == pytest.approx(20 / 2.0)


def test_single_process_is_identity():
    from paper_2112_14681_b300 import replicas
    assert replicas.max_over_ranks(None, 3.5) == 3.5
    assert replicas.aggregate_throughput(None, 4, 2.0) == (2.0, 2.0)
