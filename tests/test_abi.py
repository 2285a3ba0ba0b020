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
        if s in ("bw_set_profiling", "bw_profile_read"):
            assert hasattr(_lib.Context, s[3:]), s
        elif s in ("bw_server_submit", "bw_server_poll", "bw_server_wait", "bw_server_outstanding"):
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
