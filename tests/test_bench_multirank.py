"""The benchmark's multi-rank bookkeeping on CPU: two gloo ranks (the GPU run
uses NCCL with the same calls).  Each rank reports its own time; the job time
is the slowest rank's, and the throughput counts every rank's pixels."""
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


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local = [1.5, 2.5][rank]
    t = bench.reduce_max(local, dist, device="cpu")
    v = bench.whole_job_mpx(ws, 10, 1_000_000, t)
    q.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_time_and_weak_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in res:
        assert t == 2.5                      # slowest rank
        assert abs(v - 2 * 10 * 1.0 / 2.5) < 1e-9  # all ranks' Mpixel over that time


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(3.0, None) == 3.0
    assert bench.whole_job_mpx(1, 4, 2_000_000, 2.0) == 4.0
