"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2).

On this hardware the path is replicas only: each rank solves its own source,
the ranks meet at barriers around the timed region, and rank 0 reports the
maximum step time over ranks. These tests run that logic with two gloo ranks.
"""
import datetime
import os
import socket
import time

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank reports its own times; the max over ranks must come back
        mine = [1.0 + rank, 5.0 - rank, 0.5 * (rank + 1)]
        dist.barrier()
        got = bench.max_over_ranks(mine, dist, "cpu")
        dist.barrier()
        q.put((rank, got, bench.replica_source_seed(1, rank)))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replica_timing_is_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=100) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, got, seed in out:
        assert got == [2.0, 5.0, 1.0]
    # replicas solve different sources
    assert out[0][2] != out[1][2]


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    """Under torchrun only rank 0 runs the reference arm."""
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.main()
    assert capsys.readouterr().out == ""


def _failing_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        # the failing replica: gone between steps, before the timing reduction
        q.put((rank, "exited", 0.0))
        q.close()
        q.join_thread()
        os._exit(3)
    t0 = time.monotonic()
    try:
        bench.max_over_ranks([1.0], dist, "cpu")
        q.put((rank, "returned", time.monotonic() - t0))
    except Exception as e:  # the surviving rank learns of it on the host
        q.put((rank, type(e).__name__, time.monotonic() - t0))
    q.close()
    q.join_thread()
    os._exit(0)


@pytest.mark.timeout(120)
def test_lost_replica_ends_the_reduction_with_an_error():
    """A rank that leaves between steps: the other rank's max-over-ranks
    reduction fails within the process-group timeout instead of hanging."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert procs[1].exitcode == 3
    rank, what, secs = out[0]
    assert rank == 0 and what != "returned"
    assert secs < 60
