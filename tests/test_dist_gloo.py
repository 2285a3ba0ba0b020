"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

Each rank runs its own copy of the workload (weak scaling, no data-path
collective); the only communication is a barrier and the max-over-ranks time.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    bench.dist_init("gloo")
    r, w, lr = bench.dist_env()
    t = bench.reduce_max(1.5 + rank)
    bench.barrier()
    v = bench.weak_scaling_value(3600, 10, w, t)
    q.put((r, w, t, v))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_time_and_weak_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for r, (rank, world, t, v) in enumerate(out):
        assert rank == r and world == 2
        assert t == pytest.approx(2.5)                       # slowest rank
        assert v == pytest.approx(3600 * 10 * 2 / 2.5)        # all ranks' units / max time


def test_reference_arm_non_zero_rank_exits_without_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"]) == 0
    assert capsys.readouterr().out == ""
