"""bench.py's multi-rank path with two gloo ranks on the CPU: the barrier, the timed region
ending with its slowest rank (max over ranks), the whole-job throughput of replicas, and the
reference arm doing its work on rank 0 only."""
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _Args:
    steps = 1
    warmup = 0
    gpus = 2


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        barrier = bench.make_barrier(world)
        barrier()
        local_s = 0.5 + rank  # rank 1 is the slow one
        s = bench.max_over_ranks(local_s, world, device="cpu")
        rate = bench.whole_job_rate(1000, world, s)
        ref = bench.run_reference(_Args, world, rank) if rank != 0 else None
        barrier()
        q.put((rank, s, rate, ref))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    assert [r[0] for r in res] == [0, 1]
    for _, s, rate, ref in res:
        assert s == 1.5                      # both ranks see the slowest rank's time
        assert rate == pytest.approx(2 * 1000 / 1.5)
        assert ref is None                   # rank 1 of the reference arm returns without work


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(2.5, 1, device="cpu") == 2.5
    assert bench.whole_job_rate(300, 1, 2.0) == 150.0
    calls = []
    bench.make_barrier(1, lambda: calls.append(1))()
    assert calls == [1]
