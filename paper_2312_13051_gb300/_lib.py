"""ctypes binding of ``libberrywl.so`` (argument marshalling only).

Each function here has the name of its C entry point without the ``bw_`` prefix
and does nothing but check types, allocate the output tensors on the device and
pass pointers, sizes and the current CUDA stream through.  Every numerical step
runs in the library's kernels; without the library or a CUDA device the calls
raise instead of computing anything on the host.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libberrywl.so")

STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "EGAP", "EPSOGAP", "EWANGAP", "ENOCONV", "ETIMEOUT",
                "ECUDA", "ECANCELED"]
PRECISION = {"fp64": 0, "mixed": 1}


class BWError(RuntimeError):
    def __init__(self, code: int, msg: str, k_index: int = -1):
        name = STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else str(code)
        super().__init__(f"{name}: {msg}")
        self.code = code
        self.status = name
        self.k_index = k_index


class bw_model(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("R", C.c_void_p), ("i", C.c_void_p),
                ("j", C.c_void_p), ("t", C.c_void_p)]


class bw_plane(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("loop_dir", C.c_int32 * 3),
                ("trans_dir", C.c_double * 3), ("N", C.c_int32), ("N_t", C.c_int32)]


class bw_plane_stack(C.Structure):
    _fields_ = [("plane", bw_plane), ("sweep_dir", C.c_int32 * 3), ("N_s", C.c_int32)]


class bw_opts(C.Structure):
    _fields_ = [("gap_tol", C.c_double), ("pso_gap_tol", C.c_double),
                ("wannier_gap_tol", C.c_double), ("unitarise", C.c_int32),
                ("max_sweeps", C.c_int32), ("pso_split", C.c_int32)]


class bw_request_info(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("reserved", C.c_int32),
                ("k_index", C.c_int64), ("latency_ms", C.c_double), ("queue_ms", C.c_double),
                ("device_ms", C.c_double), ("message", C.c_char * 128)]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> C.CDLL:
    """Loads the library (raises when it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_2312_13051_gb300.build.build() first")
        lib = C.CDLL(path)
        vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "bw_create": (i32, [C.POINTER(vp), C.c_int, C.c_size_t]),
            "bw_destroy": (None, [vp]),
            "bw_last_error": (C.c_char_p, [vp]),
            "bw_get_status": (i32, [vp, vp, C.POINTER(i64)]),
            "bw_set_profiling": (i32, [vp, C.c_int]),
            "bw_profile_read": (C.c_int, [vp, C.c_int, C.c_char_p, C.POINTER(dbl)]),
            "bw_build_hk": (i32, [vp, C.POINTER(bw_model), vp, i64, C.c_int, vp, vp]),
            "bw_eigh_batched": (i32, [vp, vp, vp, i64, i32, i32, vp, vp, vp]),
            "bw_wilson_loop": (i32, [vp, C.POINTER(bw_model), C.POINTER(bw_plane), i32, i32,
                                     C.POINTER(bw_opts), vp, vp, vp]),
            "bw_nested_wilson_loop": (i32, [vp, C.POINTER(bw_model), C.POINTER(bw_plane), i32,
                                            dbl, i32, i32, i32, C.POINTER(bw_opts), vp, vp, vp,
                                            vp, vp]),
            "bw_spin_resolved_wilson_loop": (i32, [vp, C.POINTER(bw_model), C.POINTER(bw_plane),
                                                   i32, vp, i32, i32, C.POINTER(bw_opts), vp,
                                                   vp, vp, vp, vp]),
            "bw_wilson_loop_stack": (i32, [vp, C.POINTER(bw_model), C.POINTER(bw_plane_stack), i32,
                                           i32, C.POINTER(bw_opts), vp, vp, vp]),
            "bw_nested_wilson_loop_stack": (i32, [vp, C.POINTER(bw_model), C.POINTER(bw_plane_stack),
                                                  i32, dbl, i32, i32, i32, C.POINTER(bw_opts), vp,
                                                  vp, vp, vp, vp]),
            "bw_spin_resolved_wilson_loop_stack": (i32, [vp, C.POINTER(bw_model),
                                                         C.POINTER(bw_plane_stack), i32, vp, i32,
                                                         i32, C.POINTER(bw_opts), vp, vp, vp, vp,
                                                         vp]),
            "bw_winding": (i32, [vp, vp, i32, i32, vp, vp, vp]),
            "bw_z2_largest_gap": (i32, [vp, vp, i32, i32, vp, vp, vp, vp, vp]),
            "bw_plaquette_flux": (i32, [vp, C.POINTER(bw_model), C.POINTER(bw_plane), i32, vp, i32,
                                        i32, C.POINTER(bw_opts), vp, vp, vp, vp, vp]),
            "bw_wilson_loop_noalloc": (i32, [C.POINTER(bw_model), C.POINTER(bw_plane), i32, i32,
                                             C.POINTER(bw_opts), vp, vp, vp, C.c_char_p,
                                             C.c_size_t]),
            "bw_wilson_loop_workspace": (i32, [vp, C.POINTER(bw_model), C.POINTER(bw_plane), i32,
                                               i32, C.POINTER(bw_opts), C.POINTER(C.c_size_t)]),
            "bw_server_create": (i32, [C.POINTER(vp), C.c_int, i32, C.c_size_t]),
            "bw_server_destroy": (None, [vp]),
            "bw_server_last_error": (C.c_char_p, [vp]),
            "bw_server_submit": (i32, [vp, C.POINTER(bw_model), C.POINTER(bw_plane), i32, i32,
                                       C.POINTER(bw_opts), vp, vp, C.POINTER(i64)]),
            "bw_server_poll": (C.c_int, [vp, C.POINTER(bw_request_info), C.c_int]),
            "bw_server_wait": (i32, [vp, i64, dbl, C.POINTER(bw_request_info)]),
            "bw_server_outstanding": (i64, [vp]),
            "bw_server_cancel": (i32, [vp, i64]),
            "bw_selftest_unit_circle": (i32, [vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def exported_symbols():
    return ["bw_create", "bw_destroy", "bw_last_error", "bw_get_status", "bw_set_profiling",
            "bw_profile_read", "bw_build_hk",
            "bw_eigh_batched", "bw_wilson_loop", "bw_nested_wilson_loop",
            "bw_spin_resolved_wilson_loop", "bw_wilson_loop_stack", "bw_nested_wilson_loop_stack",
            "bw_spin_resolved_wilson_loop_stack", "bw_winding", "bw_z2_largest_gap", "bw_plaquette_flux", "bw_wilson_loop_noalloc", "bw_wilson_loop_workspace",
            "bw_server_create", "bw_server_destroy", "bw_server_last_error", "bw_server_submit",
            "bw_server_poll", "bw_server_wait", "bw_server_outstanding", "bw_server_cancel",
            "bw_selftest_unit_circle"]


class Context:
    """Owns one ``bw_ctx`` (device scratch arena, status word, staging buffer)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self.lib = load()
        h = C.c_void_p()
        rc = self.lib.bw_create(C.byref(h), device, mem_budget_bytes)
        if rc != 0:
            raise BWError(rc, f"bw_create(device={device}) failed")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self.lib.bw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self) -> str:
        return self.lib.bw_last_error(self.h).decode()

    def check(self, rc: int):
        if rc != 0:
            raise BWError(rc, self.error())

    def set_profiling(self, enable: bool = True) -> None:
        self.check(self.lib.bw_set_profiling(self.h, int(enable)))

    def profile_read(self, max_kernels: int = 32):
        """[(kernel name, ms)] of the most recent profiled call or graph replay."""
        names = C.create_string_buffer(32 * max_kernels)
        ms = (C.c_double * max_kernels)()
        n = self.lib.bw_profile_read(self.h, max_kernels, names, ms)
        if n < 0:
            raise BWError(8, "bw_profile_read failed")
        return [(names.raw[32 * i:32 * i + 32].split(b"\0")[0].decode(), ms[i]) for i in range(n)]

    def selftest_unit_circle(self):
        """Maximum errors of the double-float e^{2 pi i m / N}, e^{i pi t} and arg z against
        FP64 on the device (bw_selftest_unit_circle)."""
        err = (C.c_double * 3)()
        self.check(self.lib.bw_selftest_unit_circle(self.h, C.cast(err, C.c_void_p)))
        return tuple(err)

    def status(self, stream=None) -> None:
        """Synchronises the stream and raises on a device-side numerical status."""
        k = C.c_int64(-1)
        rc = self.lib.bw_get_status(self.h, _stream_ptr(stream), C.byref(k))
        if rc != 0:
            raise BWError(rc, self.error(), int(k.value))


_contexts: dict = {}


def context(device: int | None = None) -> Context:
    import torch
    if device is None:
        device = torch.cuda.current_device()
    if device not in _contexts:
        _contexts[device] = Context(device)
    return _contexts[device]


def _stream_ptr(stream=None):
    import torch
    if stream is None:
        raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        if raw is not None:  # the current stream's handle without building a Stream object
            return C.c_void_p(raw(torch.cuda.current_device()))
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


class _HostModel:
    """Keeps the contiguous host arrays of a hopping list alive during a call."""

    def __init__(self, model):
        self.R = np.ascontiguousarray(model.R, dtype=np.int32).reshape(-1, 3)
        self.i = np.ascontiguousarray(model.i, dtype=np.int32)
        self.j = np.ascontiguousarray(model.j, dtype=np.int32)
        self.t = np.ascontiguousarray(model.t, dtype=np.complex128)
        self.s = bw_model(int(model.n), int(self.t.shape[0]), self.R.ctypes.data,
                          self.i.ctypes.data, self.j.ctypes.data, self.t.ctypes.data)
        # the struct points into the caller's own arrays (no copy was made), so a later
        # call with the same arrays may reuse it; in-place edits stay visible
        self.shared = all(isinstance(b, np.ndarray) and a.ctypes.data == b.ctypes.data
                          for a, b in ((self.R, model.R), (self.i, model.i), (self.j, model.j),
                                       (self.t, model.t)))


_model_cache: dict = {}


def _host_model(model) -> _HostModel:
    """The marshalled model, reused while the model object holds the same arrays."""
    key = (id(model), id(model.R), id(model.i), id(model.j), id(model.t), int(model.n))
    hm = _model_cache.get(key)
    if hm is not None and hm.owner() is model:
        return hm
    hm = _HostModel(model)
    if hm.shared:
        import weakref
        try:
            hm.owner = weakref.ref(model)
        except TypeError:
            return hm
        if len(_model_cache) > 64:
            _model_cache.clear()
        _model_cache[key] = hm
    return hm


def _plane(plane) -> bw_plane:
    loop = [int(round(x)) for x in plane.loop_dir]
    if any(abs(float(x) - round(float(x))) > 0 for x in plane.loop_dir):
        raise BWError(1, "loop_dir must be an integer vector")
    return bw_plane((C.c_double * 3)(*map(float, plane.origin)), (C.c_int32 * 3)(*loop),
                    (C.c_double * 3)(*map(float, plane.trans_dir)), int(plane.N), int(plane.N_t))


_plane_cache: dict = {}


def _plane_arg(plane):
    """(ctypes struct, entry-point suffix, leading output shape, the single plane) for a
    plane or a stack of planes (any object with ``plane, sweep_dir, N_s``).  The struct of
    a single plane is reused for equal field values (the library only reads it)."""
    if not hasattr(plane, "sweep_dir"):
        key = (tuple(plane.origin), tuple(plane.loop_dir), tuple(plane.trans_dir), plane.N, plane.N_t)
        st = _plane_cache.get(key)
        if st is None:
            st = _plane(plane)
            if len(_plane_cache) > 256:
                _plane_cache.clear()
            _plane_cache[key] = st
        return st, "", (), plane
    sw = [int(round(x)) for x in plane.sweep_dir]
    if any(abs(float(x) - round(float(x))) > 0 for x in plane.sweep_dir):
        raise BWError(1, "sweep_dir must be an integer vector")
    st = bw_plane_stack(_plane(plane.plane), (C.c_int32 * 3)(*sw), int(plane.N_s))
    return st, "_stack", (int(plane.N_s),), plane.plane


PSO_SPLIT = {"zero": 0, "median": 1}


_default_opts = None


def _opts(gap_tol=-1.0, pso_gap_tol=-1.0, wannier_gap_tol=-1.0, unitarise=False, max_sweeps=0,
          pso_split="zero"):
    global _default_opts
    if pso_split not in PSO_SPLIT:
        raise BWError(1, f"pso_split must be one of {sorted(PSO_SPLIT)}")
    args = (float(gap_tol), float(pso_gap_tol), float(wannier_gap_tol), int(unitarise),
            int(max_sweeps), PSO_SPLIT[pso_split])
    if args == (-1.0, -1.0, -1.0, 0, 0, 0):  # the defaults: one shared, read-only struct
        if _default_opts is None:
            _default_opts = bw_opts(*args)
        return _default_opts
    return bw_opts(*args)


def _empty(shape, dtype, device):
    import torch
    return torch.empty(shape, dtype=dtype, device=device)


def _cuda_device(ctx: Context):
    import torch
    return torch.device("cuda", ctx.device)


def build_hk(model, f, complex64: bool = False, ctx: Context | None = None, check=True):
    """H(f) for each row of the device tensor ``f`` (K x 3 float64); returns K x n x n."""
    import torch
    ctx = ctx or context()
    if not (f.is_cuda and f.dtype == torch.float64 and f.is_contiguous() and f.dim() == 2
            and f.shape[1] == 3):
        raise BWError(1, "f must be a contiguous CUDA float64 tensor of shape (K, 3)")
    hm = _host_model(model)
    K = f.shape[0]
    H = _empty((K, model.n, model.n), torch.complex64 if complex64 else torch.complex128, f.device)
    ctx.check(ctx.lib.bw_build_hk(ctx.h, C.byref(hm.s), _ptr(f), K, int(complex64), _ptr(H),
                                  _stream_ptr()))
    if check:
        ctx.status()
    return H


def eigh_batched(H, n_per, n_vec: int, precision: str = "fp64", ctx: Context | None = None,
                 check=True):
    """Batched Hermitian eigensolver.  ``H``: packed complex128 CUDA tensor holding the
    matrices back to back; ``n_per``: their sizes.  Returns (evals, evecs) packed."""
    import torch
    ctx = ctx or context()
    n_per = np.ascontiguousarray(n_per, dtype=np.int32)
    if not (H.is_cuda and H.dtype == torch.complex128 and H.is_contiguous()):
        raise BWError(1, "H must be a contiguous CUDA complex128 tensor")
    if H.numel() != int(np.sum(n_per.astype(np.int64) ** 2)):
        raise BWError(1, "H size does not match n_per")
    ev = _empty((int(n_per.sum()),), torch.float64, H.device)
    vec = _empty((int(n_per.astype(np.int64).sum() * n_vec),), torch.complex128, H.device)
    ctx.check(ctx.lib.bw_eigh_batched(ctx.h, _ptr(H), n_per.ctypes.data, len(n_per), int(n_vec),
                                      PRECISION[precision], _ptr(ev),
                                      _ptr(vec) if n_vec > 0 else C.c_void_p(0), _stream_ptr()))
    if check:
        ctx.status()
    return ev, vec


def wilson_loop(model, plane, p: int, precision: str = "fp64", ctx: Context | None = None,
                check=True, out=None, **opts):
    """Hybrid Wannier centres: (phases[N_t, p], min_gap[N_t]) as CUDA float64 tensors.
    ``plane`` may be a stack of planes (``inputs.PlaneStack``): then every output has a
    leading plane axis, phases[N_s, N_t, p] and min_gap[N_s, N_t]."""
    import torch
    ctx = ctx or context()
    hm = _host_model(model)
    pl, sfx, lead, plane = _plane_arg(plane)
    o = _opts(**opts)
    if out is None:
        dev = _cuda_device(ctx)
        out = (_empty(lead + (plane.N_t, p), torch.float64, dev),
               _empty(lead + (plane.N_t,), torch.float64, dev))
    ph, gap = out
    ctx.check(getattr(ctx.lib, "bw_wilson_loop" + sfx)(
        ctx.h, C.byref(hm.s), C.byref(pl), int(p), PRECISION[precision], C.byref(o), _ptr(ph),
        _ptr(gap), _stream_ptr()))
    if check:
        ctx.status()
    return ph, gap


def nested_wilson_loop(model, plane, p: int, cut: float = -np.pi, first: int = 0,
                       m: int | None = None, precision: str = "fp64",
                       ctx: Context | None = None, check=True, out=None, **opts):
    """Nested loop: (phases[N_t, p], nested[N, m], min_wannier_gap[N_t], min_gap[N_t]);
    for a stack of planes each output has a leading plane axis (nested[N_s, N, m])."""
    import torch
    ctx = ctx or context()
    m = p // 2 if m is None else int(m)
    hm = _host_model(model)
    pl, sfx, lead, plane = _plane_arg(plane)
    o = _opts(**opts)
    if out is None:
        dev = _cuda_device(ctx)
        out = (_empty(lead + (plane.N_t, p), torch.float64, dev),
               _empty(lead + (plane.N, m), torch.float64, dev),
               _empty(lead + (plane.N_t,), torch.float64, dev),
               _empty(lead + (plane.N_t,), torch.float64, dev))
    ph, nest, wg, gap = out
    ctx.check(getattr(ctx.lib, "bw_nested_wilson_loop" + sfx)(
        ctx.h, C.byref(hm.s), C.byref(pl), int(p), float(cut), int(first), int(m),
        PRECISION[precision], C.byref(o), _ptr(ph), _ptr(nest), _ptr(wg), _ptr(gap), _stream_ptr()))
    if check:
        ctx.status()
    return ph, nest, wg, gap


def spin_resolved_wilson_loop(model, plane, p: int, spin_op, sign: int = -1,
                              precision: str = "fp64", ctx: Context | None = None, check=True,
                              want_pso=True, out=None, **opts):
    """Spin-resolved loop: (phases[N_t, p/2], pso_evals[N_t, N, p] or None,
    min_pso_gap[N_t], min_gap[N_t]); for a stack of planes each output has a leading
    plane axis."""
    import torch
    ctx = ctx or context()
    hm = _host_model(model)
    pl, sfx, lead, plane = _plane_arg(plane)
    o = _opts(**opts)
    S = np.ascontiguousarray(spin_op, dtype=np.complex128)
    if S.shape != (model.n, model.n):
        raise BWError(1, f"spin operator must be {model.n} x {model.n}")
    if out is None:
        dev = _cuda_device(ctx)
        out = (_empty(lead + (plane.N_t, p // 2), torch.float64, dev),
               _empty(lead + (plane.N_t, plane.N, p), torch.float64, dev) if want_pso else None,
               _empty(lead + (plane.N_t,), torch.float64, dev),
               _empty(lead + (plane.N_t,), torch.float64, dev))
    ph, pso, pg, gap = out
    ctx.check(getattr(ctx.lib, "bw_spin_resolved_wilson_loop" + sfx)(
        ctx.h, C.byref(hm.s), C.byref(pl), int(p), S.ctypes.data, int(sign), PRECISION[precision],
        C.byref(o), _ptr(ph), _ptr(pso), _ptr(pg), _ptr(gap), _stream_ptr()))
    if check:
        ctx.status()
    return ph, pso, pg, gap


def _need_stack(stack):
    if not hasattr(stack, "sweep_dir"):
        raise BWError(1, "expected a stack of planes (plane, sweep_dir, N_s)")


def wilson_loop_stack(model, stack, p: int, **kw):
    """``bw_wilson_loop_stack``: :func:`wilson_loop` over a stack of planes."""
    _need_stack(stack)
    return wilson_loop(model, stack, p, **kw)


def nested_wilson_loop_stack(model, stack, p: int, **kw):
    """``bw_nested_wilson_loop_stack``: :func:`nested_wilson_loop` over a stack of planes."""
    _need_stack(stack)
    return nested_wilson_loop(model, stack, p, **kw)


def spin_resolved_wilson_loop_stack(model, stack, p: int, spin_op, sign: int = -1, **kw):
    """``bw_spin_resolved_wilson_loop_stack``: :func:`spin_resolved_wilson_loop` over a
    stack of planes."""
    _need_stack(stack)
    return spin_resolved_wilson_loop(model, stack, p, spin_op, sign, **kw)


def plaquette_flux(model, plane, p: int, spin_op=None, sign: int = -1, precision: str = "fp64",
                   ctx: Context | None = None, check=True, **opts):
    """Plaquette Berry flux: (flux[N_t, N], chern scalar, min_gap[N_t], min_pso_gap[N_t]
    or None) as CUDA tensors; with ``spin_op`` the flux of the PSO sector ``sign``."""
    import torch
    ctx = ctx or context()
    dev = _cuda_device(ctx)
    hm = _host_model(model)
    pl = _plane(plane)
    o = _opts(**opts)
    S = None
    if spin_op is not None:
        S = np.ascontiguousarray(spin_op, dtype=np.complex128)
        if S.shape != (model.n, model.n):
            raise BWError(1, f"spin operator must be {model.n} x {model.n}")
    flux = _empty((plane.N_t, plane.N), torch.float64, dev)
    chern = _empty((), torch.float64, dev)
    gap = _empty((plane.N_t,), torch.float64, dev)
    pg = _empty((plane.N_t,), torch.float64, dev) if S is not None else None
    ctx.check(ctx.lib.bw_plaquette_flux(ctx.h, C.byref(hm.s), C.byref(pl), int(p),
                                        S.ctypes.data if S is not None else None, int(sign),
                                        PRECISION[precision], C.byref(o), _ptr(flux), _ptr(chern),
                                        _ptr(gap), _ptr(pg), _stream_ptr()))
    if check:
        ctx.status()
    return flux, chern, gap, pg


def winding(phases, ctx: Context | None = None, check=True, want_sums=False):
    """Winding of the summed Wannier centres of ``phases`` (CUDA float64 N_t x p) over
    the transverse grid (Eq. 6).  Returns a CUDA float64 scalar tensor, or
    (winding, sums[N_t]) with ``want_sums``."""
    import torch
    ctx = ctx or context()
    if not (phases.is_cuda and phases.dtype == torch.float64 and phases.is_contiguous()
            and phases.dim() == 2):
        raise BWError(1, "phases must be a contiguous CUDA float64 tensor of shape (N_t, p)")
    Nt, p = phases.shape
    w = _empty((), torch.float64, phases.device)
    sums = _empty((Nt,), torch.float64, phases.device) if want_sums else None
    ctx.check(ctx.lib.bw_winding(ctx.h, _ptr(phases), int(Nt), int(p), _ptr(sums), _ptr(w),
                                 _stream_ptr()))
    if check:
        ctx.status()
    return (w, sums) if want_sums else w


def z2_largest_gap(phases, ctx: Context | None = None, check=True, want_detail=False):
    """Z2 index of a time-reversal-symmetric plane from its WCC spectrum ``phases`` (CUDA
    float64 N_t x p, rows ascending, N_t even) by the largest-gap construction.  Returns
    a CUDA int32 scalar tensor (0, 1, or -1 for a rejected row), or (nu, crossings[N_t/2],
    midpoints[N_t/2 + 1], widest gaps[N_t/2 + 1]) with ``want_detail``."""
    import torch
    ctx = ctx or context()
    if not (phases.is_cuda and phases.dtype == torch.float64 and phases.is_contiguous()
            and phases.dim() == 2):
        raise BWError(1, "phases must be a contiguous CUDA float64 tensor of shape (N_t, p)")
    Nt, p = phases.shape
    dev = phases.device
    nu = _empty((), torch.int32, dev)
    h = Nt // 2
    detail = ((_empty((h,), torch.int32, dev), _empty((h + 1,), torch.float64, dev),
               _empty((h + 1,), torch.float64, dev)) if want_detail else (None, None, None))
    ctx.check(ctx.lib.bw_z2_largest_gap(ctx.h, _ptr(phases), int(Nt), int(p), _ptr(nu),
                                        *(_ptr(d) for d in detail), _stream_ptr()))
    if check:
        ctx.status()
    return (nu, *detail) if want_detail else nu


def wilson_loop_noalloc(model, plane, p: int, precision: str = "fp64", out=None, **opts):
    """``bw_wilson_loop_noalloc``: the same result as :func:`wilson_loop` computed without
    any device allocation by the library (its scratch is a fixed array inside it).
    ``out`` = (phases[N_t, p], min_gap[N_t]) caller-owned CUDA float64 tensors; when
    omitted they are allocated here, by the caller side, before the call."""
    import torch
    lib = load()
    hm = _host_model(model)
    pl = _plane(plane)
    o = _opts(**opts)
    if out is None:
        dev = torch.device("cuda", torch.cuda.current_device())
        out = (_empty((plane.N_t, p), torch.float64, dev), _empty((plane.N_t,), torch.float64, dev))
    ph, gap = out
    err = C.create_string_buffer(512)
    rc = lib.bw_wilson_loop_noalloc(C.byref(hm.s), C.byref(pl), int(p), PRECISION[precision],
                                    C.byref(o), _ptr(ph), _ptr(gap), _stream_ptr(), err, 512)
    if rc != 0:
        raise BWError(rc, err.value.decode())
    return ph, gap


def wilson_loop_workspace(model, plane, p: int, precision: str = "fp64",
                          ctx: Context | None = None, **opts) -> int:
    """Device scratch bytes ``wilson_loop`` reserves for this problem on ``ctx``."""
    ctx = ctx or context()
    hm = _host_model(model)
    pl = _plane(plane)
    o = _opts(**opts)
    nb = C.c_size_t(0)
    ctx.check(ctx.lib.bw_wilson_loop_workspace(ctx.h, C.byref(hm.s), C.byref(pl), int(p),
                                               PRECISION[precision], C.byref(o), C.byref(nb)))
    return int(nb.value)


class Server:
    """``bw_server``: memory-admitted continuous batching of Wilson-loop requests.

    ``submit`` returns a request id; the results land in host numpy arrays owned by
    this object until the request is collected with ``poll`` or ``wait``, which
    return ``(id, info, phases[N_t, p], min_gap[N_t])``.
    """

    def __init__(self, device: int = 0, max_slots: int = 4, mem_budget_bytes: int = 0):
        self.lib = load()
        h = C.c_void_p()
        rc = self.lib.bw_server_create(C.byref(h), device, int(max_slots), int(mem_budget_bytes))
        if rc != 0:
            raise BWError(rc, f"bw_server_create(device={device}) failed")
        self.h = h
        self._out = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.bw_server_destroy(self.h)
            self.h = None
            self._out.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, model, plane, p: int, precision: str = "fp64", **opts) -> int:
        hm = _host_model(model)
        pl = _plane(plane)
        o = _opts(**opts)
        ph = np.empty((plane.N_t, p), np.float64)
        gap = np.empty((plane.N_t,), np.float64)
        rid = C.c_int64(0)
        rc = self.lib.bw_server_submit(self.h, C.byref(hm.s), C.byref(pl), int(p),
                                       PRECISION[precision], C.byref(o),
                                       ph.ctypes.data_as(C.c_void_p),
                                       gap.ctypes.data_as(C.c_void_p), C.byref(rid))
        if rc != 0:
            raise BWError(rc, self.lib.bw_server_last_error(self.h).decode())
        self._out[int(rid.value)] = (ph, gap)
        return int(rid.value)

    @staticmethod
    def _info(i: bw_request_info) -> dict:
        return dict(id=int(i.id), status=STATUS_NAMES[i.status] if 0 <= i.status < len(STATUS_NAMES)
                    else str(i.status), k_index=int(i.k_index), latency_ms=i.latency_ms,
                    queue_ms=i.queue_ms, device_ms=i.device_ms, message=i.message.decode())

    def poll(self, max_requests: int = 64):
        buf = (bw_request_info * max_requests)()
        n = self.lib.bw_server_poll(self.h, buf, max_requests)
        if n < 0:
            raise BWError(1, "bw_server_poll failed")
        out = []
        for k in range(n):
            info = self._info(buf[k])
            ph, gap = self._out.pop(info["id"])
            out.append((info["id"], info, ph, gap))
        return out

    def wait(self, rid: int, timeout_s: float = 600.0):
        info = bw_request_info()
        rc = self.lib.bw_server_wait(self.h, int(rid), float(timeout_s), C.byref(info))
        if rc != 0:
            raise BWError(rc, self.lib.bw_server_last_error(self.h).decode())
        inf = self._info(info)
        ph, gap = self._out.pop(int(rid))
        return int(rid), inf, ph, gap

    def outstanding(self) -> int:
        return int(self.lib.bw_server_outstanding(self.h))

    def cancel(self, rid: int) -> None:
        """Withdraws a queued request (it completes with status ECANCELED); raises
        BWError(EINVAL) for a request already running, finished or unknown."""
        rc = self.lib.bw_server_cancel(self.h, int(rid))
        if rc != 0:
            raise BWError(rc, self.lib.bw_server_last_error(self.h).decode())
