"""GB300 space-time kernel density estimation (arXiv 1705.09366, PB-SYM hot path).

Thin ctypes binding over the C ABI in ``include/stkde.h``: the functions below
carry the C names and only marshal arguments.  Every step of the computation
runs in the CUDA library ``libstkde.so`` built from ``csrc/`` for sm_103a; if
that library is missing the binding raises instead of falling back to anything.

PyTorch (optional) supplies device memory and streams: tensors are accepted
wherever a buffer is expected, and ``stream`` may be a ``torch.cuda.Stream``.
NumPy arrays are accepted as host buffers.
"""
from __future__ import annotations

import ctypes
import os
import sys

__all__ = [
    "Options", "Grid", "Problem", "StkdeError", "Context", "lib", "lib_path",
    "stkde_default_options", "stkde_create", "stkde_compute", "stkde_compute_batch",
    "stkde_count_updates", "stkde_synchronize", "stkde_phase_times", "stkde_destroy",
    "stkde_status_string", "stkde_last_launch_count", "stkde_compute_static", "stkde_reserve",
    "stkde_inject_fault", "FORM_TENSOR_BF16X3", "FORM_TENSOR_FP16X3", "FORM_FP32", "FORM_SCATTER",
    "FORM_TENSOR_TF32X3", "FORM_TENSOR_TF32X1", "KERNEL_PRINTED", "KERNEL_UNIT_MASS",
    "FAULT_NONE", "FAULT_ALLOC", "FAULT_WITHHOLD_PAGE", "EXPORTED_SYMBOLS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "libstkde.so")

OK = 0
ERR_INVALID_ARGUMENT = 1
ERR_OOM = 2
ERR_CUDA = 3
ERR_TIMEOUT = 4
ERR_UNSUPPORTED = 5
ERR_NONFINITE = 6
ERR_INTERNAL = 7

FORM_TENSOR_BF16X3 = 0
FORM_TENSOR_FP16X3 = 1
FORM_FP32 = 2
FORM_SCATTER = 3
FORM_TENSOR_TF32X3 = 4
FORM_TENSOR_TF32X1 = 5
FORMS = {"bf16x3": FORM_TENSOR_BF16X3, "fp16x3": FORM_TENSOR_FP16X3, "fp32": FORM_FP32,
         "scatter": FORM_SCATTER, "tf32x3": FORM_TENSOR_TF32X3, "tf32x1": FORM_TENSOR_TF32X1}

KERNEL_PRINTED = 0
KERNEL_UNIT_MASS = 1

# fault injection (include/stkde_testing.h)
FAULT_NONE = 0
FAULT_ALLOC = 1
FAULT_WITHHOLD_PAGE = 2

EXPORTED_SYMBOLS = (
    "stkde_default_options", "stkde_create", "stkde_compute", "stkde_compute_batch",
    "stkde_count_updates", "stkde_synchronize", "stkde_phase_times", "stkde_destroy",
    "stkde_status_string", "stkde_last_launch_count", "stkde_compute_static",
    "stkde_compute_adaptive", "stkde_count_updates_adaptive", "stkde_abramson_bandwidths",
    "stkde_reserve", "stkde_inject_fault",
)

STATIC_MAX_EVENTS = 262144
STATIC_MAX_BINS = 1048576


class Options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("form", ctypes.c_int),
                ("kernel_constants", ctypes.c_int), ("t_block", ctypes.c_int),
                ("slab", ctypes.c_int), ("profile", ctypes.c_int)]


class Grid(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("y0", ctypes.c_double), ("t0", ctypes.c_double),
                ("sres", ctypes.c_double), ("tres", ctypes.c_double),
                ("gx", ctypes.c_int64), ("gy", ctypes.c_int64), ("gt", ctypes.c_int64)]


class Problem(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("n", ctypes.c_int64), ("grid", Grid),
                ("hs", ctypes.c_double), ("ht", ctypes.c_double), ("out", ctypes.c_void_p)]


class StkdeError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        super().__init__(f"{where}: {stkde_status_string(status)} (status {status})")


_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(lib_path):
            raise RuntimeError(f"CUDA library not built: {lib_path} is missing "
                               "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        l = ctypes.CDLL(lib_path)
        vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        l.stkde_default_options.argtypes = [ctypes.POINTER(Options)]
        l.stkde_default_options.restype = None
        l.stkde_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Options)]
        l.stkde_create.restype = ctypes.c_int
        l.stkde_compute.argtypes = [vp, vp, i64, ctypes.POINTER(Grid), dbl, dbl, vp]
        l.stkde_compute.restype = ctypes.c_int
        l.stkde_compute_batch.argtypes = [vp, ctypes.POINTER(Problem), ctypes.c_int]
        l.stkde_compute_adaptive.argtypes = [vp, vp, i64, ctypes.POINTER(Grid), vp, vp, vp]
        l.stkde_compute_adaptive.restype = ctypes.c_int
        l.stkde_count_updates_adaptive.argtypes = [vp, vp, i64, ctypes.POINTER(Grid), vp, vp,
                                                   ctypes.POINTER(ctypes.c_uint64)]
        l.stkde_count_updates_adaptive.restype = ctypes.c_int
        l.stkde_abramson_bandwidths.argtypes = [vp, vp, i64, ctypes.POINTER(Grid), dbl, dbl, dbl, dbl,
                                                dbl, vp, vp, vp]
        l.stkde_abramson_bandwidths.restype = ctypes.c_int
        l.stkde_compute_batch.restype = ctypes.c_int
        l.stkde_count_updates.argtypes = [vp, vp, i64, ctypes.POINTER(Grid), dbl, dbl,
                                          ctypes.POINTER(ctypes.c_uint64)]
        l.stkde_count_updates.restype = ctypes.c_int
        l.stkde_synchronize.argtypes = [vp]
        l.stkde_synchronize.restype = ctypes.c_int
        l.stkde_phase_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
        l.stkde_phase_times.restype = ctypes.c_int
        l.stkde_compute_static.argtypes = [vp, i64, ctypes.POINTER(Grid), dbl, dbl, vp, ctypes.c_int,
                                           ctypes.c_int, vp, ctypes.c_int]
        l.stkde_compute_static.restype = ctypes.c_int
        l.stkde_reserve.argtypes = [vp, ctypes.c_size_t]
        l.stkde_reserve.restype = ctypes.c_int
        l.stkde_inject_fault.argtypes = [vp, ctypes.c_int, i64]
        l.stkde_inject_fault.restype = ctypes.c_int
        l.stkde_last_launch_count.argtypes = [vp]
        l.stkde_last_launch_count.restype = ctypes.c_int
        l.stkde_destroy.argtypes = [vp]
        l.stkde_destroy.restype = None
        l.stkde_status_string.argtypes = [ctypes.c_int]
        l.stkde_status_string.restype = ctypes.c_char_p
        _lib = l
    return _lib


def _ptr(buf) -> int:
    """Address of a torch tensor or numpy array (0 for None / empty)."""
    if buf is None:
        return 0
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("buffer must be contiguous")
        return int(buf.data_ptr())
    if hasattr(buf, "ctypes"):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("buffer must be C-contiguous")
        return int(buf.ctypes.data) if buf.size else 0
    if isinstance(buf, int):
        return buf
    raise TypeError(f"unsupported buffer type {type(buf)!r}")


def _stream_handle(stream, device=None) -> int:
    """cudaStream_t of ``stream``: an int handle, an object with ``cuda_stream``
    (torch.cuda.Stream), or None = torch's current stream (of ``device``) when
    torch is imported and sees a GPU, else the legacy default stream (0)."""
    if stream is None:
        t = sys.modules.get("torch")
        if t is not None and t.cuda.is_available():
            return int(t.cuda.current_stream(device).cuda_stream)
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _check(st: int, where: str):
    if st != OK:
        raise StkdeError(st, where)


def stkde_status_string(status: int) -> str:
    return lib().stkde_status_string(int(status)).decode()


def stkde_default_options() -> Options:
    o = Options()
    lib().stkde_default_options(ctypes.byref(o))
    return o


def stkde_create(device: int = 0, stream=None, form="bf16x3", kernel_constants: int = 0,
                 t_block: int = 0, slab: int = 0, profile: bool = False) -> ctypes.c_void_p:
    o = stkde_default_options()
    o.device = int(device)
    o.stream = _stream_handle(stream, int(device))
    o.form = FORMS[form] if isinstance(form, str) else int(form)
    o.kernel_constants = int(kernel_constants)
    o.t_block = int(t_block)
    o.slab = int(slab)
    o.profile = int(bool(profile))
    h = ctypes.c_void_p()
    _check(lib().stkde_create(ctypes.byref(h), ctypes.byref(o)), "stkde_create")
    return h


def make_grid(gx, gy, gt, x0=0.0, y0=0.0, t0=0.0, sres=1.0, tres=1.0) -> Grid:
    return Grid(float(x0), float(y0), float(t0), float(sres), float(tres), int(gx), int(gy), int(gt))


def stkde_compute(ctx, points, n: int, grid: Grid, hs: float, ht: float, out) -> None:
    _check(lib().stkde_compute(ctx, _ptr(points), int(n), ctypes.byref(grid), float(hs),
                               float(ht), _ptr(out)), "stkde_compute")


def stkde_compute_adaptive(ctx, points, n: int, grid: Grid, hs, ht, out) -> None:
    """Per-event bandwidths: ``hs``, ``ht`` hold n float64 values each (domain
    units, host or device)."""
    _check(lib().stkde_compute_adaptive(ctx, _ptr(points), int(n), ctypes.byref(grid), _ptr(hs),
                                        _ptr(ht), _ptr(out)), "stkde_compute_adaptive")


def stkde_count_updates_adaptive(ctx, points, n: int, grid: Grid, hs, ht) -> int:
    c = ctypes.c_uint64(0)
    _check(lib().stkde_count_updates_adaptive(ctx, _ptr(points), int(n), ctypes.byref(grid),
                                              _ptr(hs), _ptr(ht), ctypes.byref(c)),
           "stkde_count_updates_adaptive")
    return int(c.value)


def stkde_abramson_bandwidths(ctx, points, n: int, grid: Grid, hs: float, ht: float, alpha: float,
                              lam_min: float, lam_max: float, pilot, hs_out, ht_out) -> None:
    _check(lib().stkde_abramson_bandwidths(ctx, _ptr(points), int(n), ctypes.byref(grid), float(hs),
                                           float(ht), float(alpha), float(lam_min), float(lam_max),
                                           _ptr(pilot), _ptr(hs_out), _ptr(ht_out)),
           "stkde_abramson_bandwidths")


def stkde_compute_batch(ctx, problems) -> None:
    arr = (Problem * len(problems))(*problems)
    _check(lib().stkde_compute_batch(ctx, arr, len(problems)), "stkde_compute_batch")


def stkde_count_updates(ctx, points, n: int, grid: Grid, hs: float, ht: float) -> int:
    c = ctypes.c_uint64(0)
    _check(lib().stkde_count_updates(ctx, _ptr(points), int(n), ctypes.byref(grid), float(hs),
                                     float(ht), ctypes.byref(c)), "stkde_count_updates")
    return int(c.value)


def stkde_synchronize(ctx) -> None:
    _check(lib().stkde_synchronize(ctx), "stkde_synchronize")


def stkde_phase_times(ctx, cap: int = 8) -> list[float]:
    buf = (ctypes.c_float * cap)()
    k = lib().stkde_phase_times(ctx, buf, cap)
    return [float(buf[i]) for i in range(k)]


def stkde_compute_static(points, n: int, grid: Grid, hs: float, ht: float, out, form="bf16x3",
                         kernel_constants: int = 0, stream=None, sync: bool = True) -> None:
    """Allocation-free density (see include/stkde.h): `points` and `out` are
    device buffers of the current device; scratch is a fixed library-owned array."""
    f = FORMS[form] if isinstance(form, str) else int(form)
    _check(lib().stkde_compute_static(_ptr(points), int(n), ctypes.byref(grid), float(hs), float(ht),
                                      _ptr(out), f, int(kernel_constants), _stream_handle(stream),
                                      int(bool(sync))), "stkde_compute_static")


def stkde_reserve(ctx, nbytes: int) -> None:
    _check(lib().stkde_reserve(ctx, int(nbytes)), "stkde_reserve")


def stkde_inject_fault(ctx, fault: int, arg: int = 0) -> None:
    """Test hook (include/stkde_testing.h): arms one injected failure on ctx."""
    _check(lib().stkde_inject_fault(ctx, int(fault), int(arg)), "stkde_inject_fault")


def stkde_last_launch_count(ctx) -> int:
    return int(lib().stkde_last_launch_count(ctx))


def stkde_destroy(ctx) -> None:
    lib().stkde_destroy(ctx)


class Context:
    """Owning wrapper of a ``stkde_ctx``.

    >>> with Context(form="bf16x3") as c:
    ...     grid = c.compute(points_cuda, (gx, gy, gt), hs, ht)   # torch.float32 on the GPU
    """

    def __init__(self, device: int = 0, stream=None, form="bf16x3", kernel_constants: int = 0,
                 t_block: int = 0, slab: int = 0, profile: bool = False):
        self.device = device
        self.handle = stkde_create(device, stream, form, kernel_constants, t_block, slab, profile)

    def close(self):
        if self.handle is not None and self.handle.value:
            stkde_destroy(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def compute(self, points, dims, hs, ht, out=None, origin=(0.0, 0.0, 0.0), sres=1.0, tres=1.0):
        """Density of ``points`` ((n, 3) float64, torch or numpy) on a grid of
        ``dims`` voxels; returns ``out`` (allocated on the device if None)."""
        gx, gy, gt = (int(d) for d in dims)
        if out is None:
            import torch
            out = torch.empty((gx, gy, gt), dtype=torch.float32, device=f"cuda:{self.device}")
        n = int(points.shape[0])
        g = make_grid(gx, gy, gt, *origin, sres=sres, tres=tres)
        stkde_compute(self.handle, points, n, g, hs, ht, out)
        return out

    def compute_adaptive(self, points, dims, hs, ht, out=None, origin=(0.0, 0.0, 0.0), sres=1.0,
                         tres=1.0):
        """Density with per-event bandwidths ``hs``, ``ht`` ((n,) float64 each,
        domain units); otherwise as :meth:`compute`."""
        gx, gy, gt = (int(d) for d in dims)
        if out is None:
            import torch
            out = torch.empty((gx, gy, gt), dtype=torch.float32, device=f"cuda:{self.device}")
        n = int(points.shape[0])
        for a in (hs, ht):
            if int(a.shape[0]) != n:
                raise ValueError("one bandwidth per event")
        g = make_grid(gx, gy, gt, *origin, sres=sres, tres=tres)
        stkde_compute_adaptive(self.handle, points, n, g, hs, ht, out)
        return out

    def count_updates_adaptive(self, points, dims, hs, ht, origin=(0.0, 0.0, 0.0), sres=1.0,
                               tres=1.0):
        g = make_grid(*dims, *origin, sres=sres, tres=tres)
        return stkde_count_updates_adaptive(self.handle, points, int(points.shape[0]), g, hs, ht)

    def abramson_bandwidths(self, points, dims, hs, ht, alpha=0.5, lam_min=0.125, lam_max=8.0,
                            pilot=None, origin=(0.0, 0.0, 0.0), sres=1.0, tres=1.0):
        """Per-event bandwidths (hs_i, ht_i) from a pilot density with the fixed pair
        (hs, ht) by Abramson's law; returns two (n,) float64 device tensors."""
        import torch
        n = int(points.shape[0])
        hs_o = torch.empty(n, dtype=torch.float64, device=f"cuda:{self.device}")
        ht_o = torch.empty(n, dtype=torch.float64, device=f"cuda:{self.device}")
        g = make_grid(*dims, *origin, sres=sres, tres=tres)
        stkde_abramson_bandwidths(self.handle, points, n, g, hs, ht, alpha, lam_min, lam_max, pilot,
                                  hs_o, ht_o)
        return hs_o, ht_o

    def compute_batch(self, problems):
        """Densities of several independent problems in one batched call.
        ``problems``: iterable of (points, dims, hs, ht, out) with device ``out``
        buffers (torch); returns the list of outputs."""
        probs, keep = [], []
        for pts, dims, hs, ht, out in problems:
            gx, gy, gt = (int(d) for d in dims)
            keep.append((pts, out))
            probs.append(Problem(_ptr(pts) if int(pts.shape[0]) > 0 else None, int(pts.shape[0]),
                                 make_grid(gx, gy, gt), float(hs), float(ht), _ptr(out)))
        stkde_compute_batch(self.handle, probs)
        return [o for _, o in keep]

    def synchronize(self):
        stkde_synchronize(self.handle)

    def count_updates(self, points, dims, hs, ht, origin=(0.0, 0.0, 0.0), sres=1.0, tres=1.0):
        g = make_grid(*dims, *origin, sres=sres, tres=tres)
        return stkde_count_updates(self.handle, points, int(points.shape[0]), g, hs, ht)

    def phase_times(self):
        return stkde_phase_times(self.handle)

    def last_launch_count(self):
        return stkde_last_launch_count(self.handle)

    def reserve(self, nbytes: int):
        """Grows the workspace now (see stkde_reserve)."""
        stkde_reserve(self.handle, nbytes)

    def inject_fault(self, fault: int, arg: int = 0):
        stkde_inject_fault(self.handle, fault, arg)
