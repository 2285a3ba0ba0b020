"""Sharding of the method's independent units over ranks (gloo, world size 2, CPU).

Rows of a plane and whole problems are split into contiguous blocks, computed per rank
and gathered on rank 0 in order.  The per-rank compute here is the FP64 oracle, so the
gathered result must equal a single-process oracle run of the whole job.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2312_13051_gb300 import inputs as I
from paper_2312_13051_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_partition_blocks():
    assert shard.partition(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert shard.partition(2, 4) == [(0, 1), (1, 2), (2, 2), (2, 2)]
    assert shard.partition(0, 2) == [(0, 0), (0, 0)]
    for n in range(0, 40):
        for w in range(1, 9):
            blocks = shard.partition(n, w)
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [e - s for s, e in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.partition(3, 0)


def test_row_block_points():
    """The rows of a block are the rows of the plane (to the last bit of rounding)."""
    plane = I.Plane(7, 11, origin=(0.1, 0.05, 0.3), trans_dir=(0.0, 1.0, 0.5))
    f = oracle.plane_points(plane)
    for i0, i1 in shard.partition(11, 3):
        fb = oracle.plane_points(shard.row_block(plane, i0, i1))
        np.testing.assert_allclose(fb, f[i0:i1], atol=1e-15, rtol=0)


def _oracle_rows(model, plane, p):
    return oracle.wilson_loop(model, plane, p)


def _nested_bbh(gamma):
    return oracle.nested_wilson_loop(I.bbh(gamma, gamma), I.Plane(8, 8), 2, m=1)[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    model = I.random_hermitian_model(6, 9)
    plane = I.Plane(9, 7)
    rows = shard.wilson_loop_rows(model, plane, 3, _oracle_rows)
    probs = shard.map_problems([0.3, 0.5, 0.9, 1.5, 2.0], _nested_bbh)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, rows, probs))


def test_two_rank_rows_and_problems_gathered_on_rank0():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        rank, rows, probs = q.get(timeout=300)
        out[rank] = (rows, probs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert out[1] == (None, None)
    rows, probs = out[0]
    ref_ph, ref_gap = oracle.wilson_loop(I.random_hermitian_model(6, 9), I.Plane(9, 7), 3)
    assert rows[0].shape == ref_ph.shape
    for r in range(ref_ph.shape[0]):
        assert oracle.circular_match_error(rows[0][r], ref_ph[r]) < 1e-12
    np.testing.assert_allclose(rows[1], ref_gap, atol=1e-12)
    want = [_nested_bbh(g) for g in (0.3, 0.5, 0.9, 1.5, 2.0)]
    assert len(probs) == len(want)
    for a, b in zip(probs, want):
        assert np.array_equal(a, b)
