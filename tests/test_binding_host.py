"""Host-side argument marshalling of the binding, on the CPU (no library calls): the
plane and option structs it reuses between calls, and the marshalled hopping list."""
import numpy as np

from paper_2312_13051_gb300 import _lib
from paper_2312_13051_gb300 import inputs as I


def test_plane_struct_reused_for_equal_planes_only():
    a = _lib._plane_arg(I.Plane(10, 12))
    b = _lib._plane_arg(I.Plane(10, 12))
    c = _lib._plane_arg(I.Plane(10, 13))
    d = _lib._plane_arg(I.Plane(10, 12, origin=(0.0, 0.0, 0.25)))
    assert a[0] is b[0]
    assert c[0] is not a[0] and d[0] is not a[0]
    assert (a[0].N, a[0].N_t) == (10, 12) and (c[0].N, c[0].N_t) == (10, 13)
    assert list(d[0].origin) == [0.0, 0.0, 0.25] and list(a[0].origin) == [0.0, 0.0, 0.0]
    assert a[1] == "" and a[2] == ()


def test_plane_stack_struct():
    st = I.PlaneStack(I.Plane(4, 6), sweep_dir=(0, 0, 1), N_s=3)
    s, sfx, lead, plane = _lib._plane_arg(st)
    assert sfx == "_stack" and lead == (3,) and plane is st.plane
    assert list(s.sweep_dir) == [0, 0, 1] and s.N_s == 3 and s.plane.N_t == 6


def test_default_options_shared_and_others_fresh():
    assert _lib._opts() is _lib._opts()
    o = _lib._opts(gap_tol=1e-3, pso_split="median")
    assert o is not _lib._opts()
    assert o.gap_tol == 1e-3 and o.pso_split == 1
    assert _lib._opts().gap_tol == -1.0 and _lib._opts().pso_split == 0


def test_marshalled_model_points_into_the_callers_arrays():
    """A model held as contiguous arrays of the ABI's types is passed without a copy,
    so edits in place reach the library (which re-plans when the list changes)."""
    m = I.bbh(0.5, 0.5)
    hm = _lib._host_model(m)
    assert hm.shared
    assert hm.s.t == m.t.ctypes.data and hm.s.R == m.R.ctypes.data
    assert _lib._host_model(m) is hm
    assert hm.s.nnz == len(m.t) and hm.s.n == m.n
    m.t[0] = m.t[0] * 1.0  # same buffer: still the same marshalled struct
    assert _lib._host_model(m).s.t == m.t.ctypes.data
    # a model whose arrays need converting is copied, and not cached
    class Loose:
        n = m.n
        R = m.R.astype(np.int64)
        i, j, t = m.i, m.j, m.t
    hl = _lib._host_model(Loose())
    assert not hl.shared and hl.s.R != m.R.ctypes.data
