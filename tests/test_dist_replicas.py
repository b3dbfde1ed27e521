"""The replica path of bench.py (one process per GPU, no data-path collective) on CPU with
gloo, world size 2: the barrier and the max-over-ranks reduction that sets the whole-job
time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench.barrier(ws)
        ms = 10.0 + 5.0 * rank                     # rank 1 is the slow replica
        worst = bench.max_over_ranks(ms, ws)
        cells = 1000
        value = ws * cells / (worst * 1e-3)        # whole-job throughput, as bench.py reports it
        out.put((rank, worst, value))
        bench.barrier(ws)
    finally:
        dist.destroy_process_group()


def test_replicas_max_over_ranks_gloo():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, worst, value in res:
        assert worst == 15.0                       # every rank sees the slowest replica
        assert abs(value - 2 * 1000 / 15e-3) < 1e-6


def test_batch_shard_partitions_grids():
    sys.path.insert(0, ROOT)
    import bench
    for ws in (1, 2, 3, 8):
        parts = [bench.shard(64, ws, r) for r in range(ws)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))                         # every grid exactly once
        assert max(map(len, parts)) - min(map(len, parts)) <= 1
