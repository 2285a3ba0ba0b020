"""The allocation-free Wilson loop against the regular entry point and the oracle.

bw_wilson_loop_noalloc exists for callers that must not have the library
allocate device memory (programs that own all device memory through their own
capped pool, plugins inside another program's CUDA context, loops that cannot
afford the synchronisation cudaMalloc / cudaFree may cause).  It runs the loop
kernels with its scratch in a fixed 8 MiB array inside the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2312_13051_gb300 import inputs as I
from tests.gpu_common import circ_err_rows, ctx, lib  # noqa: F401

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "mixed": 1e-6}
SCRATCH = 8 << 20


def _call_abi(lib, model, plane, p, precision, ph, gap):
    """Calls bw_wilson_loop_noalloc directly through the C ABI."""
    import torch
    raw = lib.load()
    hm = lib._HostModel(model)
    pl = lib._plane(plane)
    o = lib._opts()
    err = C.create_string_buffer(512)
    rc = raw.bw_wilson_loop_noalloc(C.byref(hm.s), C.byref(pl), int(p), lib.PRECISION[precision],
                                    C.byref(o), C.c_void_p(ph.data_ptr()),
                                    C.c_void_p(gap.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream), err, 512)
    return rc, err.value.decode()


def _outputs(plane, p):
    import torch
    return (torch.full((plane.N_t, p), np.nan, dtype=torch.float64, device="cuda"),
            torch.full((plane.N_t,), np.nan, dtype=torch.float64, device="cuda"))


CASES = [("bbh_60x60", lambda: (I.config_bbh().model, I.Plane(60, 60), 2)),
         ("random6_17x5", lambda: (I.random_hermitian_model(6, 2), I.Plane(17, 5), 3))]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_wilson_loop_twice(lib, ctx, precision, name, case):
    """Two calls in a row (the fixed scratch keeps the previous call's data): FP64 equal
    to bw_wilson_loop bit for bit, mixed within the mixed tolerance; both against the
    FP64 oracle within the tolerance of their precision."""
    import torch
    model, plane, p = case()
    ref_ph, ref_gap = lib.wilson_loop(model, plane, p, precision=precision, ctx=ctx)
    want, _ = oracle.wilson_loop(model, plane, p)
    for _ in range(2):
        ph, gap = _outputs(plane, p)
        rc, msg = _call_abi(lib, model, plane, p, precision, ph, gap)
        assert rc == 0, msg
        if precision == "fp64":
            assert torch.equal(ph, ref_ph)
            assert torch.equal(gap, ref_gap)
        else:
            d = torch.remainder(ph - ref_ph + np.pi, 2 * np.pi) - np.pi
            assert float(d.abs().max()) <= TOL[precision]
            assert float((gap - ref_gap).abs().max()) <= 1e-9
        assert circ_err_rows(ph.cpu().numpy(), want) <= TOL[precision]


def _bbh_bytes(K):
    """Scratch of the BBH plain loop (n = 4, p = 2; the scan kernel forms the overlaps):
    16 K n p + 8 K bytes, each rounded to 256, plus the status word and the plan."""
    al = lambda x: (x + 255) // 256 * 256
    return al(16 * K * 4 * 2) + al(8 * K)


def test_noalloc_size_limit_boundary(lib, ctx):
    """Just under the 8 MiB limit (a plane that fits only because the loop kernel forms
    the overlaps, so no K p^2 buffer is reserved) the call succeeds and equals
    bw_wilson_loop; just over it the call is refused with BW_ENOMEM before running."""
    import torch
    model = I.config_bbh().model
    under, over = I.Plane(60, 1020), I.Plane(60, 1040)
    assert _bbh_bytes(60 * 1020) + 4096 < SCRATCH < _bbh_bytes(60 * 1040)
    assert _bbh_bytes(60 * 1020) + 16 * 60 * 1020 * 4 > SCRATCH   # would not fit with overlaps
    ph, gap = _outputs(under, 2)
    rc, msg = _call_abi(lib, model, under, 2, "fp64", ph, gap)
    assert rc == 0, msg
    ref_ph, _ = lib.wilson_loop(model, under, 2, precision="fp64", ctx=ctx)
    assert torch.equal(ph, ref_ph)
    got = ph.cpu().numpy()
    for i in (0, 511, 1019):
        row = I.Plane(60, 1, origin=(0.0, i / 1020, 0.0))
        want, _ = oracle.wilson_loop(model, row, 2)
        assert oracle.circular_match_error(got[i], want[0]) <= TOL["fp64"]
    ph, gap = _outputs(over, 2)
    rc, msg = _call_abi(lib, model, over, 2, "fp64", ph, gap)
    assert lib.STATUS_NAMES[rc] == "ENOMEM", msg
    assert "fixed scratch" in msg
    assert bool(torch.isnan(ph).all())       # nothing ran


def test_noalloc_reports_device_status(lib):
    plane = I.Plane(8, 8)          # the Eq. 4 gap closes at (pi, pi) for m = 2
    ph, gap = _outputs(plane, 1)
    rc, msg = _call_abi(lib, I.chern_eq4(2.0), plane, 1, "fp64", ph, gap)
    assert lib.STATUS_NAMES[rc] == "EGAP", msg
    rc, msg = _call_abi(lib, I.chern_eq4(1.5), plane, 1, "fp64", ph, gap)   # cleared per call
    assert rc == 0, msg
