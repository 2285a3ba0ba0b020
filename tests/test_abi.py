"""The C ABI library builds for sm_103a, loads, and exports every declared symbol.

Runs without a GPU: no compute call is made.  Without a CUDA device bw_create()
must fail with BW_ECUDA instead of falling back to the host.
"""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "berrywl.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bw_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2312_13051_gb300 import build
    return build.build()


def test_header_declares_the_paper_entry_points():
    syms = declared_symbols()
    for name in ("bw_build_hk", "bw_eigh_batched", "bw_wilson_loop", "bw_nested_wilson_loop",
                 "bw_spin_resolved_wilson_loop", "bw_create", "bw_destroy", "bw_get_status",
                 "bw_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    from paper_2312_13051_gb300 import _lib
    assert sorted(_lib.exported_symbols()) == declared_symbols()
    for s in declared_symbols():
        if s in ("bw_set_profiling", "bw_profile_read", "bw_selftest_unit_circle"):
            assert hasattr(_lib.Context, s[3:]), s
        elif s in ("bw_server_submit", "bw_server_poll", "bw_server_wait", "bw_server_outstanding",
                   "bw_server_cancel"):
            assert hasattr(_lib.Server, s[len("bw_server_"):]), s
        elif s not in ("bw_create", "bw_destroy", "bw_last_error", "bw_get_status",
                       "bw_server_create", "bw_server_destroy", "bw_server_last_error"):
            assert hasattr(_lib, s[3:]), s


def test_no_device_fails_loudly(libpath):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2312_13051_gb300 import _lib
    with pytest.raises(_lib.BWError) as e:
        _lib.Context(0)
    assert e.value.status == "ECUDA"


def test_model_marshalling_cache():
    """The binding reuses the marshalled hopping list only while the model object holds
    the same arrays: reassigned arrays are marshalled again, in-place edits stay
    visible (the struct points at the caller's memory), copies are never cached."""
    import numpy as np
    from paper_2312_13051_gb300 import _lib, inputs as I
    m = I.bbh(0.5, 0.5)
    a = _lib._host_model(m)
    assert a.shared and _lib._host_model(m) is a and a.s.t == m.t.ctypes.data
    m.t[0] = 7.0
    assert _lib._host_model(m) is a
    m.t = m.t * 2
    b = _lib._host_model(m)
    assert b is not a and b.s.t == m.t.ctypes.data
    m.i = m.i.astype(np.int64)                 # needs a copy: marshalled every call
    c = _lib._host_model(m)
    assert not c.shared and _lib._host_model(m) is not c


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structures have the C compiler's size and field offsets for
    every struct the header defines (a layout slip would pass garbage silently)."""
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if not gcc:
        pytest.skip("no C compiler")
    from paper_2312_13051_gb300 import _lib
    structs = [_lib.bw_model, _lib.bw_plane, _lib.bw_plane_stack, _lib.bw_opts, _lib.bw_request_info]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "berrywl.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f in st._fields_:
            lines.append(f'  printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, c = line.split()
        got[(a, b)] = int(c)
    for st in structs:
        name = st.__name__
        assert got[(name, "sizeof")] == ctypes.sizeof(st), name
        for f in st._fields_:
            assert got[(name, f[0])] == getattr(st, f[0]).offset, (name, f[0])


def test_plane_stack_marshalling():
    """A stack of planes: plane s at origin + (s / N_s) sweep_dir; the binding passes the
    first plane, the integer sweep and N_s, refuses a fractional sweep, and gives its
    outputs a leading plane axis."""
    from paper_2312_13051_gb300 import _lib, inputs as I
    st = I.PlaneStack(I.Plane(8, 6, origin=(0.1, 0.0, 0.25)), (0, 0, 1), 4)
    origins = [pl.origin for pl in st.planes()]
    assert origins == [(0.1, 0.0, 0.25), (0.1, 0.0, 0.5), (0.1, 0.0, 0.75), (0.1, 0.0, 1.0)]
    assert all(pl.N == 8 and pl.N_t == 6 for pl in st.planes())
    s, sfx, lead, base = _lib._plane_arg(st)
    assert sfx == "_stack" and lead == (4,) and base is st.plane
    assert list(s.sweep_dir) == [0, 0, 1] and s.N_s == 4 and s.plane.N_t == 6
    assert list(s.plane.origin) == [0.1, 0.0, 0.25]
    s1, sfx1, lead1, _ = _lib._plane_arg(st.plane)
    assert sfx1 == "" and lead1 == () and s1.N == 8
    with pytest.raises(_lib.BWError):
        _lib._plane_arg(I.PlaneStack(st.plane, (0, 0, 0.5), 2))
