"""Shared fixtures and comparison helpers for the GPU tests."""
import numpy as np
import pytest

import oracle


def circ_err_rows(got, ref):
    """Max over rows of the circular match error between sorted phase lists."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    return max(oracle.circular_match_error(got[r], ref[r]) for r in range(got.shape[0]))


@pytest.fixture(scope="session")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_13051_gb300 import build as b
    b.build()
    from paper_2312_13051_gb300 import _lib
    _lib.load()
    return _lib


@pytest.fixture(scope="session")
def ctx(lib):
    c = lib.Context(0)
    yield c
    c.close()
