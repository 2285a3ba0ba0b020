"""Failure detection without a GPU fault.

Every failure here is made on the host (a non-finite amplitude, a budget that is too
small, a request withdrawn from the server's queue) or by a bounded device loop that
runs out (an eigensolver given one Jacobi sweep): the kernels return a status the host
reads, and the context stays usable afterwards.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2312_13051_gb300 import inputs as I
from tests.gpu_common import circ_err_rows, ctx, lib  # noqa: F401

pytestmark = pytest.mark.gpu
P = I.Plane


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_jacobi_sweep_cap_reports_enoconv(lib, ctx, precision):
    """A dense random n = 12 model needs several Jacobi sweeps: with max_sweeps = 1 the
    shared-memory solver stops after one and the call reports BW_ENOCONV with the
    failing k-point; the next call on the same context is unaffected."""
    model = I.random_hermitian_model(12, 4)
    plane = P(6, 4)
    with pytest.raises(lib.BWError) as e:
        lib.wilson_loop(model, plane, 5, precision=precision, ctx=ctx, max_sweeps=1)
    assert e.value.status == "ENOCONV"
    assert 0 <= e.value.k_index < plane.N * plane.N_t
    ph, _ = lib.wilson_loop(model, plane, 5, precision=precision, ctx=ctx)
    ref, _ = oracle.wilson_loop(model, plane, 5)
    assert circ_err_rows(ph.cpu().numpy(), ref) <= (1e-10 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_amplitude_is_rejected(lib, ctx, bad):
    """A NaN or infinite hopping amplitude is refused on the host (BW_EINVAL naming the
    hopping) before anything is uploaded or launched."""
    m = I.bbh(0.5, 0.5)
    t = m.t.copy()
    t[3] = complex(bad, 0.0)
    model = I.HoppingList(n=m.n, R=m.R, i=m.i, j=m.j, t=t, dim=m.dim)
    with pytest.raises(lib.BWError) as e:
        lib.wilson_loop(model, P(8, 8), 2, ctx=ctx)
    assert e.value.status == "EINVAL"
    assert "non-finite" in str(e.value)


def test_budget_too_small_reports_enomem(lib):
    """A context with an 8 MiB scratch budget refuses a 160 000 k-point plane (its
    occupied states alone take 20 MB) with BW_ENOMEM, then runs a problem that fits."""
    small = lib.Context(0, mem_budget_bytes=8 << 20)
    try:
        model = I.config_bbh().model
        with pytest.raises(lib.BWError) as e:
            lib.wilson_loop(model, P(400, 400), 2, ctx=small)
        assert e.value.status == "ENOMEM"
        assert "budget" in str(e.value)
        ph, _ = lib.wilson_loop(model, P(12, 12), 2, ctx=small)
        ref, _ = oracle.wilson_loop(model, P(12, 12), 2)
        assert circ_err_rows(ph.cpu().numpy(), ref) <= 1e-10
    finally:
        small.close()


def test_server_cancel_queued_request(lib):
    """With one slot, a request submitted behind a long one stays queued; cancelling it
    completes it at once with status ECANCELED, the long one finishes normally, and
    cancelling a running or collected request is refused."""
    srv = lib.Server(0, max_slots=1)
    try:
        big = I.supercell(I.spin_hall(1.0), 10, W=2.0, seed=5)       # n = 400, p = 200
        r1 = srv.submit(big, P(16, 16), 200, "fp64")
        r2 = srv.submit(I.bbh(0.5, 0.5), P(8, 8), 2, "fp64")
        srv.cancel(r2)
        _, info2, _, _ = srv.wait(r2, 5.0)
        assert info2["status"] == "ECANCELED", info2
        time.sleep(0.05)              # the worker admits r1 within a millisecond
        if srv.outstanding():         # r1 is on the GPU (its solve takes ~0.7 s)
            with pytest.raises(lib.BWError) as e:
                srv.cancel(r1)
            assert e.value.status == "EINVAL"
        _, info1, ph, _ = srv.wait(r1, 300.0)
        assert info1["status"] == "OK", info1
        row = P(16, 1, origin=(0.0, 3 / 16, 0.0))
        ref, _ = oracle.wilson_loop(big, row, 200)
        assert oracle.circular_match_error(ph[3], ref[0]) <= 1e-10
        with pytest.raises(lib.BWError):
            srv.cancel(r1)
    finally:
        srv.close()
