"""Thin Python binding of the ebsdxcf C ABI (include/ebsdxcf.h).

Argument marshalling only: every step runs in the CUDA library
``_build/libebsdxcf.so``.  Functions carry the C names; tensors are torch CUDA
tensors (device pointers) except for the ``*_host`` entry point, which takes
CPU tensors.  Work is enqueued on torch's current CUDA stream.  If the library
is missing or cannot be loaded, every call raises; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

XCF_OK = 0
XCF_ERR_ARG = -1
XCF_ERR_SIZE = -2
XCF_ERR_OOM = -3
XCF_ERR_CUDA = -4
XCF_ERR_TIMEOUT = -5
XCF_ERR_UNIMPLEMENTED = -6
XCF_NOALLOC_SCRATCH_BYTES = 16 << 20   # size of xcf_index_noalloc's fixed array


class XcfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class xcf_options(C.Structure):
    _fields_ = [("window", C.c_int32), ("sigma_hp", C.c_double), ("sigma_lp", C.c_double),
                ("lp_nr", C.c_int32), ("lp_neta", C.c_int32), ("lp_rmin", C.c_double),
                ("lp_rmax", C.c_double), ("max_iter", C.c_int32), ("tol_deg", C.c_double),
                ("upsample", C.c_int32), ("master_interp", C.c_int32), ("ndp_bg_sigma", C.c_double),
                ("lp_windows", C.c_int32), ("native_sizes", C.c_int32)]


class xcf_geometry(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("pcx", C.c_double),
                ("pcy", C.c_double), ("pcz", C.c_double), ("sample_tilt_deg", C.c_double),
                ("detector_tilt_deg", C.c_double)]


def geometry(width, height, pc=(0.5, 0.5, 0.6), sample_tilt=70.0, detector_tilt=0.0) -> xcf_geometry:
    return xcf_geometry(int(width), int(height), float(pc[0]), float(pc[1]), float(pc[2]),
                        float(sample_tilt), float(detector_tilt))


_P = C.c_void_p
_I32 = C.c_int32


class xcf_map_desc(C.Structure):
    _fields_ = [("lib", _P), ("patterns", _P), ("P", _I32), ("best", _P), ("peak", _P), ("shift", _P)]


# name -> (argtypes, restype)
_SIGS = {
    "xcf_strerror": ([C.c_int], C.c_char_p),
    "xcf_last_error": ([_P], C.c_char_p),
    "xcf_options_default": ([C.POINTER(xcf_options)], C.c_int),
    "xcf_crop": ([C.POINTER(xcf_geometry), C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32),
                  C.POINTER(C.c_double)], C.c_int),
    "xcf_crop_ex": ([C.POINTER(xcf_geometry), _I32, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32),
                     C.POINTER(C.c_double)], C.c_int),
    "xcf_create": ([C.POINTER(_P), C.POINTER(xcf_options), C.c_int], C.c_int),
    "xcf_destroy": ([_P], C.c_int),
    "xcf_project": ([_P, _P, _I32, _P, _I32, C.POINTER(xcf_geometry), _P, _P, _P], C.c_int),
    "xcf_prep": ([_P, _P, _I32, C.POINTER(xcf_geometry), _P, _P, _P, _P], C.c_int),
    "xcf_build_library": ([_P, _P, _I32, _P, _I32, C.POINTER(xcf_geometry), C.POINTER(_P), _P], C.c_int),
    "xcf_build_library_images": ([_P, _P, _P, _I32, C.POINTER(xcf_geometry), _P, _I32, C.POINTER(_P),
                                  _P], C.c_int),
    "xcf_library_free": ([_P], C.c_int),
    "xcf_library_info": ([_P, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_P)], C.c_int),
    "xcf_index": ([_P, _P, _P, _I32, _P, _P, _P, _P, _P], C.c_int),
    "xcf_correlate_all": ([_P, _P, _P, _I32, _P, _P], C.c_int),
    "xcf_refine": ([_P, _P, _P, _I32, _P, _P, _I32, C.c_double, _P, _P, _P, _P], C.c_int),
    "xcf_disorientation": ([_P, _P, _P, _I32, _P, _P], C.c_int),
    "xcf_index_refine_host": ([_P, _P, _P, _I32, _P, _I32, _P, _P, _P, _P, _P, _P], C.c_int),
    "xcf_index_refine": ([_P, _P, _P, _I32, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "xcf_build_library_ex": ([_P, _P, _I32, _P, _I32, C.POINTER(xcf_geometry), _P, _I32, C.POINTER(_P), _P],
                             C.c_int),
    "xcf_screen_topk": ([_P, _P, _P, _I32, _I32, _P, _P, _P], C.c_int),
    "xcf_rescore": ([_P, _P, _P, _I32, _P, _I32, _P, _P, _P, _P], C.c_int),
    "xcf_refine_best": ([_P, _P, _P, _I32, _P, _P, _P, _P, _P, _P], C.c_int),
    "xcf_index_precision": ([_P, _P, _P, _I32, _P, _I32, _P, _P, _P, _P, _P], C.c_int),
    "xcf_index_ndp": ([_P, _P, _P, _I32, _I32, _P, _P, _P, _P, _P], C.c_int),
    "xcf_rotation_scan": ([_P, _P, _I32, _P, _P, _P, _I32, C.c_double, _P, _P, _P, _P], C.c_int),
    "xcf_net_set_bf16": ([_P, _I32], C.c_int),
    "xcf_so3_grid": ([_P, C.c_double, _I32, _P, C.c_int64, _P, _P], C.c_int),
    "xcf_nearest_disorientation": ([_P, _P, _I32, _P, _I32, _I32, _P, _P, _P], C.c_int),
    "xcf_index_noalloc": ([_P, _P, _P, _I32, _P, _P, _P, _P], C.c_int),
    "xcf_noalloc_max_patterns": ([_I32], C.c_int),
    "xcf_index_maps": ([_P, _P, _I32, _I32, _P], C.c_int),
    "xcf_maps_get_tuning": ([_P, _I32, _I32, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32)], C.c_int),
    "xcf_maps_set_tuning": ([_P, _I32, _I32, _I32, _I32, _I32], C.c_int),
    "xcf_net_num_params": ([_I32], C.c_int64),
    "xcf_net_create": ([_P, _I32, _P, C.POINTER(_P)], C.c_int),
    "xcf_net_free": ([_P], C.c_int),
    "xcf_net_params": ([_P, C.POINTER(_P), C.POINTER(C.c_int64)], C.c_int),
    "xcf_net_forward": ([_P, _P, _P, _I32, C.POINTER(xcf_geometry), _P, _P], C.c_int),
    "xcf_net_loss_grad": ([_P, _P, _P, _I32, C.POINTER(xcf_geometry), _P, _P, _P, _P, _P], C.c_int),
    "xcf_net_adam": ([_P, _P, C.c_float, C.c_float, C.c_float, C.c_float, _P], C.c_int),
    "xcf_propose": ([_P, _P, _P, _I32, C.POINTER(xcf_geometry), _P, _P], C.c_int),
    "xcf_index_learned": ([_P, _P, _P, _P, _I32, _P, C.c_float, _P, _P, _P, _P, _P], C.c_int),
    "xcf_fp32_fma_rate": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_double), _P], C.c_int),
    "xcf_set_scratch_limit": ([_P, C.c_uint64], C.c_int),
    "xcf_scratch_bytes": ([_P, C.POINTER(C.c_uint64)], C.c_int),
    "xcf_profile_enable": ([_P, C.c_int], C.c_int),
    "xcf_profile_read": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int], C.c_int),
}

STAGES = ("project", "prep", "search", "peak", "logpolar", "update", "other", "screen", "net")

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if asked and needed)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"ebsdxcf CUDA library not built: {path}")
        lib = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc: int, ctx=None):
    if rc != XCF_OK:
        lib = load()
        detail = lib.xcf_last_error(ctx).decode() if ctx else ""
        raise XcfError(rc, f"{lib.xcf_strerror(rc).decode()}: {detail}")


def _ptr(t, dtype, name, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _hptr(t, dtype, name, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if t.dtype != dtype or t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CPU {dtype} tensor")
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


_PER_PATTERN = {"patterns": None, "best": 1, "peak": 1, "shift": 2, "pcs": 3, "seeds": 4, "quats": 4,
                "iters": 1, "rpeak": 1, "peaks": 0}


def _sizes(lib, P, **tensors):
    """Element counts of a call's tensors against P and the library's
    detector: patterns must hold exactly P x H x W values and every other
    tensor at least P times its per-pattern count (an undersized output would
    be written out of bounds on the device)."""
    for name, t in tensors.items():
        if t is None:
            continue
        per = _PER_PATTERN[name]
        if per is None:
            want = P * lib.geom.width * lib.geom.height
            if t.numel() != want:
                raise ValueError(f"{name} holds {t.numel()} values, expected {P} x {lib.geom.height} x "
                                 f"{lib.geom.width} = {want}")
        elif name == "peaks":
            if t.numel() < P * lib.T:
                raise ValueError(f"peaks holds {t.numel()} values, expected at least {P} x {lib.T}")
        elif t.numel() < P * per:
            raise ValueError(f"{name} holds {t.numel()} values, expected at least {P} x {per}")


# ------------------------------------------------------------------ handles
class Context:
    """An xcf_ctx on one CUDA device (owns reusable device scratch)."""

    def __init__(self, options: xcf_options | None = None, device: int | None = None, **kw):
        lib = load()
        o = xcf_options()
        lib.xcf_options_default(C.byref(o))
        if options is not None:
            o = options
        for k, v in kw.items():
            setattr(o, k, v)
        self.options = o
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = C.c_void_p()
        _check(lib.xcf_create(C.byref(h), C.byref(o), self.device))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load().xcf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Library:
    """An xcf_library (device-resident template spectra)."""

    def __init__(self, handle, geom: xcf_geometry, quats: torch.Tensor | None = None):
        self.handle = handle
        self.geom = geom
        T, N, sp = _I32(), _I32(), C.c_void_p()
        _check(load().xcf_library_info(handle, C.byref(T), C.byref(N), C.byref(sp)))
        self.T, self.N, self._spectra_ptr = T.value, N.value, sp.value
        self.quats = quats

    def spectra(self) -> torch.Tensor:
        """Copy of the library's half spectra [T, N, N/2+1] complex64."""
        shape = (self.T, self.N, self.N // 2 + 1, 2)

        class _View:
            __cuda_array_interface__ = {"shape": shape, "typestr": "<f4", "version": 3,
                                        "data": (self._spectra_ptr, False), "strides": None}
        view = torch.as_tensor(_View(), device=f"cuda:{torch.cuda.current_device()}")
        return torch.view_as_complex(view.clone())

    def close(self):
        if getattr(self, "handle", None):
            load().xcf_library_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ entry points
def xcf_crop(geom: xcf_geometry, native: bool = False):
    n, ox, oy = _I32(), _I32(), _I32()
    pc = (C.c_double * 3)()
    _check(load().xcf_crop_ex(C.byref(geom), int(bool(native)), C.byref(n), C.byref(ox), C.byref(oy), pc))
    return n.value, ox.value, oy.value, tuple(pc)


def xcf_project(ctx: Context, master, quats, geom: xcf_geometry, pcs=None, out=None):
    P = quats.shape[0]
    if out is None:
        out = torch.empty((P, geom.height, geom.width), dtype=torch.float32, device=quats.device)
    _check(load().xcf_project(ctx.handle, _ptr(master, torch.float32, "master"), master.shape[-1],
                              _ptr(quats, torch.float64, "quats"), P, C.byref(geom),
                              _ptr(pcs, torch.float64, "pcs", True), _ptr(out, torch.float32, "out"),
                              _stream()), ctx.handle)
    return out


def xcf_prep(ctx: Context, images, geom: xcf_geometry, want_spatial=False):
    P = images.shape[0]
    n = xcf_crop(geom, ctx.options.native_sizes)[0]
    spec = torch.empty((P, n, n // 2 + 1, 2), dtype=torch.float32, device=images.device)
    spat = torch.empty((P, n, n), dtype=torch.float32, device=images.device) if want_spatial else None
    degen = torch.empty(P, dtype=torch.int32, device=images.device)
    _check(load().xcf_prep(ctx.handle, _ptr(images, torch.float32, "images"), P, C.byref(geom),
                           _ptr(spec, torch.float32, "spectra"), _ptr(spat, torch.float32, "spatial", True),
                           _ptr(degen, torch.int32, "degenerate"), _stream()), ctx.handle)
    return torch.view_as_complex(spec), spat, degen


def xcf_build_library(ctx: Context, master, quats, geom: xcf_geometry) -> Library:
    h = C.c_void_p()
    _check(load().xcf_build_library(ctx.handle, _ptr(master, torch.float32, "master"), master.shape[-1],
                                    _ptr(quats, torch.float64, "quats"), quats.shape[0], C.byref(geom),
                                    C.byref(h), _stream()), ctx.handle)
    return Library(h, geom, quats)


def xcf_build_library_images(ctx: Context, images, quats, geom: xcf_geometry, master=None) -> Library:
    h = C.c_void_p()
    M = master.shape[-1] if master is not None else 0
    _check(load().xcf_build_library_images(ctx.handle, _ptr(images, torch.float32, "images"),
                                           _ptr(quats, torch.float64, "quats"), quats.shape[0],
                                           C.byref(geom), _ptr(master, torch.float32, "master", True), M,
                                           C.byref(h), _stream()), ctx.handle)
    return Library(h, geom, quats)


def xcf_index(ctx: Context, lib: Library, patterns, best=None, peak=None, shift=None, pcs=None):
    """pcs: per-pattern pattern centres [P, 3] float64 (None: the library's)."""
    P = patterns.shape[0]
    dev = patterns.device
    best = torch.empty(P, dtype=torch.int32, device=dev) if best is None else best
    peak = torch.empty(P, dtype=torch.float32, device=dev) if peak is None else peak
    shift = torch.empty((P, 2), dtype=torch.float32, device=dev) if shift is None else shift
    _sizes(lib, P, patterns=patterns, best=best, peak=peak, shift=shift, pcs=pcs)
    _check(load().xcf_index(ctx.handle, lib.handle, _ptr(patterns, torch.float32, "patterns"), P,
                            _ptr(pcs, torch.float64, "pcs", True),
                            _ptr(best, torch.int32, "best"), _ptr(peak, torch.float32, "peak"),
                            _ptr(shift, torch.float32, "shift"), _stream()), ctx.handle)
    return best, peak, shift


def xcf_correlate_all(ctx: Context, lib: Library, patterns, peaks=None):
    P = patterns.shape[0]
    peaks = torch.empty((P, lib.T), dtype=torch.float32, device=patterns.device) if peaks is None else peaks
    _sizes(lib, P, patterns=patterns, peaks=peaks)
    _check(load().xcf_correlate_all(ctx.handle, lib.handle, _ptr(patterns, torch.float32, "patterns"), P,
                                    _ptr(peaks, torch.float32, "peaks"), _stream()), ctx.handle)
    return peaks


def xcf_refine(ctx: Context, lib: Library, patterns, seeds, pcs=None, quats=None, peak=None, iters=None,
               max_iter=0, tol_deg=-1.0):
    """max_iter <= 0 / tol_deg < 0: the context's options."""
    P = patterns.shape[0]
    dev = patterns.device
    quats = torch.empty((P, 4), dtype=torch.float64, device=dev) if quats is None else quats
    peak = torch.empty(P, dtype=torch.float32, device=dev) if peak is None else peak
    iters = torch.empty(P, dtype=torch.int32, device=dev) if iters is None else iters
    _sizes(lib, P, patterns=patterns, seeds=seeds, pcs=pcs, quats=quats, peak=peak, iters=iters)
    _check(load().xcf_refine(ctx.handle, lib.handle, _ptr(patterns, torch.float32, "patterns"), P,
                             _ptr(seeds, torch.float64, "seeds"), _ptr(pcs, torch.float64, "pcs", True),
                             int(max_iter), float(tol_deg),
                             _ptr(quats, torch.float64, "quats"), _ptr(peak, torch.float32, "peak"),
                             _ptr(iters, torch.int32, "iters"), _stream()), ctx.handle)
    return quats, peak, iters


def xcf_disorientation(ctx: Context, qa, qb, out=None):
    n = qa.shape[0]
    out = torch.empty(n, dtype=torch.float64, device=qa.device) if out is None else out
    _check(load().xcf_disorientation(ctx.handle, _ptr(qa, torch.float64, "qa"), _ptr(qb, torch.float64, "qb"),
                                     n, _ptr(out, torch.float64, "out"), _stream()), ctx.handle)
    return out


def xcf_index_refine(ctx: Context, lib: Library, patterns, pcs=None, out=None):
    """Search + refinement in one call on device tensors; returns a dict of outputs."""
    P = patterns.shape[0]
    d = patterns.device
    if out is None:
        out = dict(best=torch.empty(P, dtype=torch.int32, device=d), peak=torch.empty(P, device=d),
                   shift=torch.empty((P, 2), device=d), quats=torch.empty((P, 4), dtype=torch.float64, device=d),
                   rpeak=torch.empty(P, device=d), iters=torch.empty(P, dtype=torch.int32, device=d))
    _sizes(lib, P, patterns=patterns, pcs=pcs, **out)
    _check(load().xcf_index_refine(
        ctx.handle, lib.handle, _ptr(patterns, torch.float32, "patterns"), P, _ptr(pcs, torch.float64, "pcs", True),
        _ptr(out["best"], torch.int32, "best"), _ptr(out["peak"], torch.float32, "peak"),
        _ptr(out["shift"], torch.float32, "shift"), _ptr(out["quats"], torch.float64, "quats"),
        _ptr(out["rpeak"], torch.float32, "rpeak"), _ptr(out["iters"], torch.int32, "iters"), _stream()),
        ctx.handle)
    return out


def xcf_index_refine_host(ctx: Context, lib: Library, patterns, pcs=None, chunk=0, out=None):
    """Host-memory end to end (synchronous); patterns [P, H, W] CPU float32 (pinned for speed)."""
    P = patterns.shape[0]
    if out is None:
        pin = patterns.is_pinned()
        mk = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=pin)
        out = dict(best=mk((P,), torch.int32), peak=mk((P,), torch.float32), shift=mk((P, 2), torch.float32),
                   quats=mk((P, 4), torch.float64), rpeak=mk((P,), torch.float32), iters=mk((P,), torch.int32))
    _sizes(lib, P, patterns=patterns, pcs=pcs, **out)
    _check(load().xcf_index_refine_host(
        ctx.handle, lib.handle, _hptr(patterns, torch.float32, "patterns"), P,
        _hptr(pcs, torch.float64, "pcs", True), int(chunk), _hptr(out["best"], torch.int32, "best"),
        _hptr(out["peak"], torch.float32, "peak"), _hptr(out["shift"], torch.float32, "shift"),
        _hptr(out["quats"], torch.float64, "quats"), _hptr(out["rpeak"], torch.float32, "rpeak"),
        _hptr(out["iters"], torch.int32, "iters")), ctx.handle)
    return out


def xcf_fp32_fma_rate(ctx: Context):
    """Measured FP32 FMA throughput of the device -> (TFLOP/s, ms per launch)."""
    t, ms = C.c_double(), C.c_double()
    _check(load().xcf_fp32_fma_rate(ctx.handle, C.byref(t), C.byref(ms), _stream()), ctx.handle)
    return t.value, ms.value


def xcf_set_scratch_limit(ctx: Context, nbytes: int):
    _check(load().xcf_set_scratch_limit(ctx.handle, int(nbytes)), ctx.handle)


def xcf_scratch_bytes(ctx: Context) -> int:
    b = C.c_uint64()
    _check(load().xcf_scratch_bytes(ctx.handle, C.byref(b)), ctx.handle)
    return int(b.value)


def xcf_profile_enable(ctx: Context, on: bool = True):
    _check(load().xcf_profile_enable(ctx.handle, 1 if on else 0), ctx.handle)


def xcf_profile_read(ctx: Context, reset: bool = False):
    """-> {stage: (device_ms, launches)}"""
    ms = (C.c_double * len(STAGES))()
    n = (C.c_int64 * len(STAGES))()
    _check(load().xcf_profile_read(ctx.handle, ms, n, 1 if reset else 0), ctx.handle)
    return {s: (ms[i], n[i]) for i, s in enumerate(STAGES)}


def xcf_noalloc_max_patterns(n: int) -> int:
    return int(load().xcf_noalloc_max_patterns(int(n)))


def xcf_index_noalloc(ctx: Context, lib: Library, patterns, best, peak, shift):
    """xcf_index without any device allocation by the library (its scratch is
    a fixed array compiled into the library).  Outputs must be preallocated."""
    P = patterns.shape[0]
    _sizes(lib, P, patterns=patterns, best=best, peak=peak, shift=shift)
    _check(load().xcf_index_noalloc(ctx.handle, lib.handle, _ptr(patterns, torch.float32, "patterns"), P,
                                    _ptr(best, torch.int32, "best"), _ptr(peak, torch.float32, "peak"),
                                    _ptr(shift, torch.float32, "shift"), _stream()), ctx.handle)
    return best, peak, shift


XCF_LIB_SCREEN = 1
XCF_LIB_NDP = 2
XCF_LIB_NO_SPECTRA = 4


def xcf_build_library_ex(ctx: Context, quats, geom: xcf_geometry, master=None, images=None, flags: int = 0) -> Library:
    """Library from the master (images None) or from template images; flags
    XCF_LIB_SCREEN keeps BF16 filtered images for xcf_screen_topk, XCF_LIB_NDP
    the contrast-normalised FP32 + BF16 images for xcf_index_ndp,
    XCF_LIB_NO_SPECTRA skips the FFT spectra (no correlation search)."""
    h = C.c_void_p()
    M = master.shape[-1] if master is not None else 0
    _check(load().xcf_build_library_ex(ctx.handle, _ptr(master, torch.float32, "master", True), M,
                                       _ptr(quats, torch.float64, "quats"), quats.shape[0], C.byref(geom),
                                       _ptr(images, torch.float32, "images", True), int(flags), C.byref(h),
                                       _stream()), ctx.handle)
    return Library(h, geom, quats)


def xcf_screen_topk(ctx: Context, lib: Library, patterns, k: int = 32):
    """-> (cand [P, k] int32, score [P, k] float32): BF16 zero-shift screen on the tensor cores."""
    P = patterns.shape[0]
    cand = torch.empty((P, k), dtype=torch.int32, device=patterns.device)
    score = torch.empty((P, k), dtype=torch.float32, device=patterns.device)
    _check(load().xcf_screen_topk(ctx.handle, lib.handle, _ptr(patterns, torch.float32, "patterns"), P, int(k),
                                  _ptr(cand, torch.int32, "cand"), _ptr(score, torch.float32, "score"), _stream()),
           ctx.handle)
    return cand, score


def xcf_index_ndp(ctx: Context, lib: Library, patterns, k: int = 4, want_cand: bool = False):
    """Dictionary indexing by the normalised dot product (Eq. 1): BF16
    tensor-core NDP over the library, FP32 rescore of the k best.
    -> (best [P] int32, ndp [P] float32) or, with want_cand, also
    (cand [P, k] int32, cand_score [P, k] float32)."""
    P, d = patterns.shape[0], patterns.device
    best = torch.empty(P, dtype=torch.int32, device=d)
    ndp = torch.empty(P, dtype=torch.float32, device=d)
    cand = torch.empty((P, k), dtype=torch.int32, device=d) if want_cand else None
    cs = torch.empty((P, k), dtype=torch.float32, device=d) if want_cand else None
    _check(load().xcf_index_ndp(ctx.handle, lib.handle, _ptr(patterns, torch.float32, "patterns"), P, int(k),
                                _ptr(best, torch.int32, "best"), _ptr(ndp, torch.float32, "ndp"),
                                _ptr(cand, torch.int32, "cand", True), _ptr(cs, torch.float32, "cand_score", True),
                                _stream()), ctx.handle)
    return (best, ndp, cand, cs) if want_cand else (best, ndp)


def xcf_rotation_scan(ctx: Context, master, geom: xcf_geometry, q, h: int, step_deg: float, pc_test=None):
    """Peak-width experiment (Figs. 3, 4): reference of orientation q [4]
    against the crystal rotated about detector x, y, z by (j - h) step_deg.
    -> (ndp [3, 2h+1], xcf [3, 2h+1], fwhm [2, 3] degrees, -1 unresolved)."""
    d = master.device
    L = 2 * int(h) + 1
    ndp = torch.empty((3, L), dtype=torch.float32, device=d)
    xc = torch.empty((3, L), dtype=torch.float32, device=d)
    fw = torch.empty((2, 3), dtype=torch.float32, device=d)
    _check(load().xcf_rotation_scan(ctx.handle, _ptr(master, torch.float32, "master"), master.shape[-1],
                                    C.byref(geom), _ptr(q, torch.float64, "q"),
                                    _ptr(pc_test, torch.float64, "pc_test", True), int(h), float(step_deg),
                                    _ptr(ndp, torch.float32, "ndp"), _ptr(xc, torch.float32, "xcf"),
                                    _ptr(fw, torch.float32, "fwhm"), _stream()), ctx.handle)
    return ndp, xc, fw


XCF_SO3_DEDUP = 1


def xcf_so3_grid(ctx: Context, step_deg: float, dedup: bool = True, device=None):
    """S^2 x S^1 library orientations in the cubic fundamental zone -> [T, 4] float64 (device)."""
    d = torch.device("cuda", ctx.device) if device is None else device
    n = C.c_int64()
    flags = XCF_SO3_DEDUP if dedup else 0
    _check(load().xcf_so3_grid(ctx.handle, float(step_deg), flags, None, 0, C.byref(n), _stream()), ctx.handle)
    q = torch.empty((n.value, 4), dtype=torch.float64, device=d)
    _check(load().xcf_so3_grid(ctx.handle, float(step_deg), flags, _ptr(q, torch.float64, "quats"), n.value,
                               C.byref(n), _stream()), ctx.handle)
    return q


def xcf_nearest_disorientation(ctx: Context, qa, qb=None, mode: int | None = None):
    """Nearest qb of each qa under the cubic disorientation -> (angle_deg [na] float64, index [na] int32).
    qb None: qa against itself without self (mode 1); mode 2: earlier entries only."""
    na = qa.shape[0]
    if mode is None:
        mode = 1 if qb is None else 0
    ang = torch.empty(na, dtype=torch.float64, device=qa.device)
    idx = torch.empty(na, dtype=torch.int32, device=qa.device)
    _check(load().xcf_nearest_disorientation(ctx.handle, _ptr(qa, torch.float64, "qa"), na,
                                             _ptr(qb, torch.float64, "qb", True), qb.shape[0] if qb is not None else 0,
                                             int(mode), _ptr(ang, torch.float64, "angle"),
                                             _ptr(idx, torch.int32, "index"), _stream()), ctx.handle)
    return ang, idx


def xcf_refine_best(ctx: Context, lib: Library, patterns, best, pcs=None, out=None):
    """Refinement seeded by the library orientations of best -> (quats, peak, iters)."""
    P = patterns.shape[0]
    d = patterns.device
    if out is None:
        out = (torch.empty((P, 4), dtype=torch.float64, device=d), torch.empty(P, device=d),
               torch.empty(P, dtype=torch.int32, device=d))
    q, pk, it = out
    _sizes(lib, P, patterns=patterns, best=best, pcs=pcs, quats=q, peak=pk, iters=it)
    _check(load().xcf_refine_best(ctx.handle, lib.handle, _ptr(patterns, torch.float32, "patterns"), P,
                                  _ptr(best, torch.int32, "best"), _ptr(pcs, torch.float64, "pcs", True),
                                  _ptr(q, torch.float64, "quats"), _ptr(pk, torch.float32, "peak"),
                                  _ptr(it, torch.int32, "iters"), _stream()), ctx.handle)
    return q, pk, it


def xcf_rescore(ctx: Context, lib: Library, patterns, cand):
    """FP32 FFT cross-correlation against each pattern's candidates -> (best, peak, shift)."""
    P, k = cand.shape
    d = patterns.device
    best = torch.empty(P, dtype=torch.int32, device=d)
    peak = torch.empty(P, dtype=torch.float32, device=d)
    shift = torch.empty((P, 2), dtype=torch.float32, device=d)
    _check(load().xcf_rescore(ctx.handle, lib.handle, _ptr(patterns, torch.float32, "patterns"), P,
                              _ptr(cand, torch.int32, "cand"), int(k), _ptr(best, torch.int32, "best"),
                              _ptr(peak, torch.float32, "peak"), _ptr(shift, torch.float32, "shift"), _stream()),
           ctx.handle)
    return best, peak, shift


XCF_MAPS_GRAPH = 1


XCF_BODY_REG, XCF_BODY_ROUNDS, XCF_BODY_SMEM, XCF_BODY_OCT = 0, 1, 2, 3


def xcf_maps_get_tuning(ctx: Context, N: int, T: int):
    """-> (body, groups, pairs) chosen for side N and library size T, or None if not tuned yet."""
    b, g, p = _I32(), _I32(), _I32()
    rc = load().xcf_maps_get_tuning(ctx.handle, int(N), int(T), C.byref(b), C.byref(g), C.byref(p))
    return (b.value, g.value, p.value) if rc == XCF_OK else None


def xcf_maps_set_tuning(ctx: Context, N: int, T: int, body: int, pairs: int, groups: int = 1):
    _check(load().xcf_maps_set_tuning(ctx.handle, int(N), int(T), int(body), int(groups), int(pairs)), ctx.handle)


def xcf_index_maps(ctx: Context, maps, outs=None, graph: bool = False):
    """Index several maps (each a (Library, patterns [P, H, W]) pair, detectors
    of any supported size) with one persistent search launch.  With graph=True
    the batch is captured as a CUDA graph and replayed while the same tensors
    (patterns and outputs, pass `outs` back in) are given.  -> outs, a list of
    (best, peak, shift) per map."""
    n = len(maps)
    if outs is None:
        outs = []
        for lib, pats in maps:
            P, d = pats.shape[0], pats.device
            outs.append((torch.empty(P, dtype=torch.int32, device=d), torch.empty(P, dtype=torch.float32, device=d),
                         torch.empty((P, 2), dtype=torch.float32, device=d)))
    desc = (xcf_map_desc * max(n, 1))()
    for i, ((lib, pats), (best, peak, shift)) in enumerate(zip(maps, outs)):
        _sizes(lib, pats.shape[0], patterns=pats, best=best, peak=peak, shift=shift)
        desc[i] = xcf_map_desc(lib.handle, _ptr(pats, torch.float32, "patterns"), pats.shape[0],
                               _ptr(best, torch.int32, "best"), _ptr(peak, torch.float32, "peak"),
                               _ptr(shift, torch.float32, "shift"))
    _check(load().xcf_index_maps(ctx.handle, C.cast(desc, _P), n, XCF_MAPS_GRAPH if graph else 0, _stream()),
           ctx.handle)
    return outs


# ------------------------------------------------------- proposal network
def xcf_net_num_params(k: int = 8) -> int:
    return int(load().xcf_net_num_params(int(k)))


class Net:
    """Proposal network handle (parameters and Adam state on the device)."""

    def __init__(self, handle, k: int):
        self.handle, self.k = handle, k
        p, n = C.c_void_p(), C.c_int64()
        _check(load().xcf_net_params(handle, C.byref(p), C.byref(n)))
        self.n, self._ptr = n.value, p.value

    def params(self):
        """Writable device view of the parameters (float32 [n])."""
        class _View:
            pass
        v = _View()
        v.__cuda_array_interface__ = {"shape": (self.n,), "typestr": "<f4", "data": (self._ptr, False),
                                      "version": 3, "strides": None}
        return torch.as_tensor(v, device="cuda")

    def set_bf16(self, on: bool = True):
        """Inference forward with BF16 tensor-core convolutions (True) or FP32 (False)."""
        _check(load().xcf_net_set_bf16(self.handle, 1 if on else 0))

    def close(self):
        if getattr(self, "handle", None):
            load().xcf_net_free(self.handle)
            self.handle = None

    __del__ = close


def _geom_ref(geom):
    return C.byref(geom) if geom is not None else None


def xcf_net_create(ctx: Context, k: int = 8, params=None) -> Net:
    h = C.c_void_p()
    _check(load().xcf_net_create(ctx.handle, int(k), _ptr(params, torch.float32, "params", True), C.byref(h)),
           ctx.handle)
    return Net(h, int(k))


def xcf_net_forward(ctx: Context, net: Net, images, geom: xcf_geometry | None = None):
    B = images.shape[0]
    out = torch.empty((B, 6 * net.k), dtype=torch.float32, device=images.device)
    _check(load().xcf_net_forward(ctx.handle, net.handle, _ptr(images, torch.float32, "images"), B, _geom_ref(geom),
                                  _ptr(out, torch.float32, "out"), _stream()), ctx.handle)
    return out


def xcf_net_loss_grad(ctx: Context, net: Net, images, quats_gt, geom: xcf_geometry | None = None,
                      want_grad: bool = False, want_winners: bool = False):
    """-> (loss [1] float64 device tensor, grad [n] or None, winners [B, 2] or None)"""
    B, d = images.shape[0], images.device
    loss = torch.empty(1, dtype=torch.float64, device=d)
    grad = torch.empty(net.n, dtype=torch.float32, device=d) if want_grad else None
    win = torch.empty((B, 2), dtype=torch.int32, device=d) if want_winners else None
    _check(load().xcf_net_loss_grad(ctx.handle, net.handle, _ptr(images, torch.float32, "images"), B,
                                    _geom_ref(geom), _ptr(quats_gt, torch.float64, "quats_gt"),
                                    _ptr(loss, torch.float64, "loss"), _ptr(grad, torch.float32, "grad", True),
                                    _ptr(win, torch.int32, "winners", True), _stream()), ctx.handle)
    return loss, grad, win


def xcf_net_adam(ctx: Context, net: Net, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8):
    _check(load().xcf_net_adam(ctx.handle, net.handle, lr, beta1, beta2, eps, _stream()), ctx.handle)


def xcf_propose(ctx: Context, net: Net, patterns, geom: xcf_geometry | None = None):
    """-> quats [P, k, 4] float64"""
    P = patterns.shape[0]
    q = torch.empty((P, net.k, 4), dtype=torch.float64, device=patterns.device)
    _check(load().xcf_propose(ctx.handle, net.handle, _ptr(patterns, torch.float32, "patterns"), P, _geom_ref(geom),
                              _ptr(q, torch.float64, "quats"), _stream()), ctx.handle)
    return q


def xcf_index_learned(ctx: Context, net: Net, lib: Library, patterns, pcs=None, tau: float = 0.3, out=None):
    """Proposals -> correlation score -> refinement, with the full search as
    fallback below tau.  -> (quats [P, 4], peak [P], iters [P], fallback [P])"""
    P, d = patterns.shape[0], patterns.device
    if out is None:
        out = (torch.empty((P, 4), dtype=torch.float64, device=d), torch.empty(P, dtype=torch.float32, device=d),
               torch.empty(P, dtype=torch.int32, device=d), torch.empty(P, dtype=torch.int32, device=d))
    q, pk, it, fb = out
    _check(load().xcf_index_learned(ctx.handle, net.handle, lib.handle, _ptr(patterns, torch.float32, "patterns"), P,
                                    _ptr(pcs, torch.float64, "pcs", True), float(tau), _ptr(q, torch.float64, "quats"),
                                    _ptr(pk, torch.float32, "peak"), _ptr(it, torch.int32, "iters"),
                                    _ptr(fb, torch.int32, "fallback"), _stream()), ctx.handle)
    return out


def xcf_index_precision(ctx: Context, lib: Library, patterns, pcs=None, k: int = 32, out=None):
    """Screen top-k + FP32 rescore + refinement with one pre-processing of the
    patterns.  -> (best [P], quats [P, 4], peak [P], iters [P])"""
    P, d = patterns.shape[0], patterns.device
    if out is None:
        out = (torch.empty(P, dtype=torch.int32, device=d), torch.empty((P, 4), dtype=torch.float64, device=d),
               torch.empty(P, dtype=torch.float32, device=d), torch.empty(P, dtype=torch.int32, device=d))
    b, q, pk, it = out
    _check(load().xcf_index_precision(ctx.handle, lib.handle, _ptr(patterns, torch.float32, "patterns"), P,
                                      _ptr(pcs, torch.float64, "pcs", True), int(k), _ptr(b, torch.int32, "best"),
                                      _ptr(q, torch.float64, "quats"), _ptr(pk, torch.float32, "peak"),
                                      _ptr(it, torch.int32, "iters"), _stream()), ctx.handle)
    return out
