"""The oracle's per-row nested-loop work spread over host processes (test helper).

Large oracle references (thousands of n = 256 eigensolves) take minutes in one
process.  The oracle's nested loop maps a per-row task over the transverse rows;
this helper runs those tasks in a process pool started with ``spawn`` (safe after
CUDA has been initialised in the parent).  The model goes to each worker once,
through the pool initialiser, instead of once per row.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import oracle
import oracle.wilson as OW

_W = {}


def _init(common):
    _W["common"] = common
    model = common[0]
    _W["blocks"] = oracle.translation_blocks(model)


def _row(i):
    model, plane, p, gap_tol, bases, cut, first, m, wtol, unitarise = _W["common"]
    return OW._nested_row_task((model, plane, i, p, gap_tol, bases, cut, first, m, wtol, unitarise,
                                _W["blocks"]))


def nested_wilson_loop(model, plane, p, cut, first, m, bases, workers=None, gap_tol=None,
                       wannier_gap_tol=1e-6, timeout_s=600.0):
    """``oracle.nested_wilson_loop`` for the given base points, rows in parallel (H(f)
    from the per-translation blocks)."""
    gap_tol = 1e-6 * max(1.0, float(abs(model.t).max())) if gap_tol is None else gap_tol
    common = (model, plane, p, gap_tol, list(bases), cut, first, m, wannier_gap_tol, False)
    workers = workers or max(1, min(os.cpu_count() or 1, plane.N_t))
    # one BLAS thread per worker process (the workers fill the cores); spawned workers
    # read these variables when they import numpy
    saved = {k: os.environ.get(k) for k in _BLAS_VARS}
    os.environ.update({k: "1" for k in _BLAS_VARS})
    try:
        return _run(model, plane, p, cut, first, m, bases, workers, gap_tol, wannier_gap_tol,
                    timeout_s, common)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


_BLAS_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _run(model, plane, p, cut, first, m, bases, workers, gap_tol, wannier_gap_tol, timeout_s, common):
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                initializer=_init, initargs=(common,)) as ex:
        def row_map(_fn, tasks):
            # bounded: a pool whose workers cannot start must fail, not wait forever
            return ex.map(_row, [t[2] for t in tasks], chunksize=1, timeout=timeout_s)
        return oracle.nested_wilson_loop(model, plane, p, cut=cut, first=first, m=m,
                                         gap_tol=gap_tol, wannier_gap_tol=wannier_gap_tol,
                                         bases=bases, row_map=row_map)
