"""Parity at the full sizes of the benchmark configurations, on sampled outputs.

The GPU runs the whole plane in the launch configuration the bench uses; the oracle
recomputes selected transverse rows (each row is an independent loop), or the
whole plane where that takes seconds.
"""
import numpy as np
import pytest

import oracle
from paper_2312_13051_gb300 import inputs as I
from tests.gpu_common import circ_err_rows, ctx, lib  # noqa: F401

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-6}


def _row_plane(plane, i):
    return I.Plane(plane.N, 1, origin=tuple(np.array(plane.origin) + np.array(plane.trans_dir) * i / plane.N_t),
                   loop_dir=plane.loop_dir, trans_dir=plane.trans_dir)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_manyband_full_size_sampled_rows(lib, ctx, precision):
    """n = 256, p = 64 on the 101 x 101 grid (10 201 k-points, waves of 2048)."""
    wl = I.config_manyband()
    ph, gap = lib.wilson_loop(wl.model, wl.plane, wl.p, precision=precision, ctx=ctx)
    ph, gap = ph.cpu().numpy(), gap.cpu().numpy()
    for i in (0, 50, 100):
        ref, rgap = oracle.wilson_loop(wl.model, _row_plane(wl.plane, i), wl.p)
        assert oracle.circular_match_error(ph[i], ref[0]) <= TOL[precision]
        assert abs(gap[i] - rgap[0]) <= 1e-6 * max(1.0, abs(rgap[0]))


def test_manyband_full_size_spin_sampled_rows(lib, ctx):
    wl = I.config_manyband()
    ph, pso, _, _ = lib.spin_resolved_wilson_loop(wl.model, wl.plane, wl.p, wl.spin_op, -1,
                                                  precision="mixed", ctx=ctx)
    ph, pso = ph.cpu().numpy(), pso.cpu().numpy()
    for i in (17, 83):
        ref, rpso, _, _ = oracle.spin_resolved_wilson_loop(wl.model, _row_plane(wl.plane, i), wl.p,
                                                           wl.spin_op, -1)
        assert oracle.circular_match_error(ph[i], ref[0]) <= TOL["mixed"]
        # The mixed PSO eigenvalues are FP64 Rayleigh quotients of FP32 Jacobi vectors:
        # error ~ theta^2 Delta, with Delta the spacing inside the +-1 clusters (down to
        # ~2e-5 here) and theta ~ 5e-7 / Delta the mixing left by the FP32 stopping test,
        # i.e. ~(5e-7)^2 / Delta ~ 1e-8.  The sector's span (what the phases use) is
        # Newton-refined separately.
        d = np.abs(pso.reshape(wl.plane.N_t, wl.plane.N, wl.p)[i] - rpso.reshape(wl.plane.N, wl.p)).max()
        assert d <= 1e-7, d


def test_disordered_supercell_L10_full_plane(lib, ctx):
    """Config 2 at L = 10 (n = 400, p = 200), one realisation, the whole 16 x 16 plane."""
    wl = I.config_disordered(10, seed=20231213 + 2)
    ref, rgap = oracle.wilson_loop(wl.model, wl.plane, wl.p)
    for precision in ("mixed", "fp64"):
        ph, gap = lib.wilson_loop(wl.model, wl.plane, wl.p, precision=precision, ctx=ctx)
        assert circ_err_rows(ph.cpu().numpy(), ref) <= TOL[precision]


_L20 = {}


def _l20_reference(wl, i):
    if i not in _L20:
        _L20[i] = oracle.wilson_loop(wl.model, _row_plane(wl.plane, i), wl.p)[0][0]
    return _L20[i]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_disordered_supercell_L20_sampled_row(lib, ctx, precision):
    """Config 2 at L = 20 (n = 1600, p = 800): whole plane on the GPU, one row checked."""
    wl = I.config_disordered(20, seed=20231213 + 5)
    ph, _ = lib.wilson_loop(wl.model, wl.plane, wl.p, precision=precision, ctx=ctx)
    i = 5
    assert oracle.circular_match_error(ph.cpu().numpy()[i], _l20_reference(wl, i)) <= TOL[precision]


_MB_NESTED = {}


def _manyband_nested_reference(wl, bases):
    key = tuple(bases)
    if key not in _MB_NESTED:
        from tests import oracle_pool
        _MB_NESTED[key] = oracle_pool.nested_wilson_loop(wl.model, wl.plane, wl.p, -np.pi, 0,
                                                         wl.nested_m, bases)
    return _MB_NESTED[key]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_manyband_full_size_nested_sampled_bases(lib, ctx, precision):
    """Config 3's nested loop at full size (n = 256, p = 64, lower half m = 32 of the
    Wannier bands, 101 x 101): the GPU runs the whole plane in one call; the oracle
    (rows spread over host processes) gives the first-loop phases of every row and the
    nested phases of three base points."""
    wl = I.config_manyband()
    bases = (0, 37, 88)
    ph, nest, wgap, _ = lib.nested_wilson_loop(wl.model, wl.plane, wl.p, m=wl.nested_m,
                                               precision=precision, ctx=ctx)
    ref_ph, ref_nest, ref_wgap, _ = _manyband_nested_reference(wl, bases)
    assert circ_err_rows(ph.cpu().numpy(), ref_ph) <= TOL[precision]
    nest = nest.cpu().numpy()
    for b, j in enumerate(bases):
        assert oracle.circular_match_error(nest[j], ref_nest[b]) <= TOL[precision], j
    # the GPU reports the gap per row over every base point; the oracle over three
    assert float(wgap.min()) <= ref_wgap + 1e-9


def test_serving_requests_sampled(lib):
    """Config-4 requests (flux supercells, L in {8, 12}) through the server."""
    reqs = [r for r in I.serving_requests(40) if r["L"] in (8, 12)][:3]
    srv = lib.Server(0, max_slots=3)
    try:
        ids = []
        for r in reqs:
            m = I.serving_model(r)
            ids.append((srv.submit(m, I.Plane(r["nk"], r["nk"]), m.n // 2, "mixed"), m, r))
        for rid, m, r in ids:
            _, info, ph, _ = srv.wait(rid, 300)
            assert info["status"] == "OK", info
            pl = I.Plane(r["nk"], r["nk"])
            i = r["nk"] // 3
            ref, _ = oracle.wilson_loop(m, _row_plane(pl, i), m.n // 2)
            assert oracle.circular_match_error(ph[i], ref[0]) <= TOL["mixed"]
    finally:
        srv.close()
