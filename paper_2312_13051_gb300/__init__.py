"""GB300 (sm_103a) Wilson-loop library: hybrid, nested and spin-resolved Wannier centres.

The compute path is ``libberrywl.so`` (hand-written CUDA kernels behind a C ABI);
this package holds its ctypes binding, the build helper and the seeded input
generators.  Importing the package does not load the library; the first call does,
and fails loudly when the library or a CUDA device is missing.
"""

_API = ("build_hk", "eigh_batched", "wilson_loop", "nested_wilson_loop",
        "spin_resolved_wilson_loop", "Context", "BWError", "context")


def __getattr__(name):
    if name in _API:
        from . import _lib
        return getattr(_lib, name)
    raise AttributeError(name)


__all__ = list(_API)
