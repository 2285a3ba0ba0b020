"""Request server (continuous batching): every result is the same alone and in the mix.

Requests of different sizes (small-n, tridiagonal and p > 64 paths, both precisions)
run concurrently on the server's slots; each result must equal, bit for bit, the
same request run alone through ``wilson_loop``, and match the oracle.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2312_13051_gb300 import inputs as I
from tests.gpu_common import circ_err_rows, ctx, lib  # noqa: F401

pytestmark = pytest.mark.gpu

P = I.Plane


def _mix():
    """(model, plane, p, precision) for a mix of flux supercells and one primitive cell."""
    reqs = []
    for k, (L, nk, prec) in enumerate([(2, 5, "fp64"), (3, 4, "mixed"), (4, 6, "fp64"),
                                       (6, 4, "mixed"), (2, 7, "mixed"), (3, 3, "fp64"),
                                       (6, 3, "fp64"), (4, 5, "mixed")]):
        m = I.supercell(I.spin_hall(1.0), L, W=1.0 + 0.3 * k, seed=100 + k, flux=True)
        reqs.append((m, P(nk, nk - 1), m.n // 2, prec))
    reqs.append((I.spin_hall(1.0), P(9, 6), 2, "fp64"))
    return reqs


def test_server_mix_equals_alone(lib, ctx):
    reqs = _mix()
    srv = lib.Server(0, max_slots=3)
    try:
        ids = [srv.submit(m, pl, p, prec) for (m, pl, p, prec) in reqs]
        got = {}
        t0 = time.time()
        while len(got) < len(ids):
            for rid, info, ph, gap in srv.poll():
                assert info["status"] == "OK", info
                got[rid] = (ph, gap, info)
            assert time.time() - t0 < 300, "server did not finish"
            time.sleep(0.002)
        assert srv.outstanding() == 0
    finally:
        srv.close()
    for rid, (m, pl, p, prec) in zip(ids, reqs):
        ph, gap, info = got[rid]
        assert info["latency_ms"] >= info["queue_ms"] >= 0.0
        alone, galone = lib.wilson_loop(m, pl, p, precision=prec, ctx=ctx)
        assert np.array_equal(ph, alone.cpu().numpy()), (m.name, prec)
        assert np.array_equal(gap, galone.cpu().numpy()), (m.name, prec)
    m, pl, p, prec = reqs[3]                       # n = 144, p = 72 (GEMM loop path), mixed
    ref, _ = oracle.wilson_loop(m, pl, p)
    assert circ_err_rows(got[ids[3]][0], ref) <= 1e-6


def test_server_small_request_overtakes_large(lib):
    """A small request submitted after a large one finishes first: it is admitted
    while the large one runs and its kernels overlap with it."""
    big = I.supercell(I.spin_hall(1.0), 8, W=2.0, seed=9, flux=True)   # n = 256, p = 128
    small = I.spin_hall(1.0)
    srv = lib.Server(0, max_slots=2)
    try:
        a = srv.submit(big, P(10, 10), 128, "fp64")
        b = srv.submit(small, P(6, 6), 2, "fp64")
        order = []
        t0 = time.time()
        while len(order) < 2:
            order += [rid for rid, info, _, _ in srv.poll()]
            assert time.time() - t0 < 300
            time.sleep(0.001)
        assert order == [b, a]
    finally:
        srv.close()


def test_server_reports_device_status_and_continues(lib):
    """A closed gap (odd p on the doubly degenerate spin-Hall bands) comes back as
    EGAP for that request only; the next request on the same slot is unaffected."""
    srv = lib.Server(0, max_slots=1)
    try:
        bad = srv.submit(I.spin_hall(1.0), P(5, 4), 3, "fp64")
        good = srv.submit(I.spin_hall(1.0), P(5, 4), 2, "fp64")
        _, ib, _, _ = srv.wait(bad, 60)
        _, ig, ph, _ = srv.wait(good, 60)
        assert ib["status"] == "EGAP" and ib["k_index"] >= 0
        assert ig["status"] == "OK"
        ref, _ = oracle.wilson_loop(I.spin_hall(1.0), P(5, 4), 2)
        assert circ_err_rows(ph, ref) <= 1e-10
        with pytest.raises(lib.BWError):
            srv.submit(I.spin_hall(1.0), P(5, 4), 5, "fp64")        # p > n
    finally:
        srv.close()
