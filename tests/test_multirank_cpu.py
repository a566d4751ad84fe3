"""The multi-rank path of bench.py ("replicas only": every rank multiplies its
own copy, the job figure is all ranks' flops over the slowest rank's time),
run as world-size-2 gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate_ranks(1.0 + rank, 1e9 * (rank + 1), world, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, value))


def test_replicas_take_max_time_and_sum_flops():
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
    # slowest rank: 2.0 ms; total flops 1e9 + 2e9 -> 3e9 / 2e-3 s = 1500 GFLOP/s on every rank
    for rank, ms, value in out:
        assert ms == 2.0
        assert abs(value - 1500.0) < 1e-9


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.aggregate_ranks(0.5, 1e9, 1)
    assert ms == 0.5 and abs(value - 2000.0) < 1e-9
