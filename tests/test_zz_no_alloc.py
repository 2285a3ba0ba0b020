"""The allocation-free Wilson loop against the regular entry point.

bw_wilson_loop_noalloc exists for callers that must not have the library
allocate device memory (programs that own all device memory through their own
capped pool, plugins inside another program's CUDA context, loops that cannot
afford the synchronisation cudaMalloc / cudaFree may cause).  It runs the same
kernels with its scratch in a fixed array inside the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2312_13051_gb300 import inputs as I
from tests.gpu_common import ctx, lib  # noqa: F401

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "mixed": 1e-6}


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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_wilson_loop_twice(lib, ctx, precision):
    import torch
    cases = [(I.config_bbh().model, I.Plane(60, 60), 2),
             (I.random_hermitian_model(6, 2), I.Plane(17, 5), 3)]
    for model, plane, p in cases:
        ref_ph, ref_gap = lib.wilson_loop(model, plane, p, precision=precision, ctx=ctx)
        for _ in range(2):          # the fixed scratch keeps the previous call's data
            ph = torch.full((plane.N_t, p), np.nan, dtype=torch.float64, device="cuda")
            gap = torch.full((plane.N_t,), np.nan, dtype=torch.float64, device="cuda")
            rc, msg = _call_abi(lib, model, plane, p, precision, ph, gap)
            assert rc == 0, msg
            d = torch.remainder(ph - ref_ph + np.pi, 2 * np.pi) - np.pi
            assert float(d.abs().max()) <= TOL[precision]
            assert float((gap - ref_gap).abs().max()) <= 1e-9


def test_noalloc_rejects_oversized_problem(lib):
    import torch
    plane = I.Plane(400, 400)      # 160000 k-points x 4 x 2 complex128: beyond 8 MiB
    ph = torch.empty((plane.N_t, 2), dtype=torch.float64, device="cuda")
    gap = torch.empty((plane.N_t,), dtype=torch.float64, device="cuda")
    rc, msg = _call_abi(lib, I.config_bbh().model, plane, 2, "fp64", ph, gap)
    assert lib.STATUS_NAMES[rc] == "ENOMEM"
    assert "fixed scratch" in msg


def test_noalloc_reports_device_status(lib):
    import torch
    plane = I.Plane(8, 8)          # the Eq. 4 gap closes at (pi, pi) for m = 2
    ph = torch.empty((plane.N_t, 1), dtype=torch.float64, device="cuda")
    gap = torch.empty((plane.N_t,), dtype=torch.float64, device="cuda")
    rc, msg = _call_abi(lib, I.chern_eq4(2.0), plane, 1, "fp64", ph, gap)
    assert lib.STATUS_NAMES[rc] == "EGAP", msg
    rc, msg = _call_abi(lib, I.chern_eq4(1.5), plane, 1, "fp64", ph, gap)   # cleared per call
    assert rc == 0, msg
