"""FP64 CPU oracle of the refined template-matching EBSD indexer (arXiv 1807.11313).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The arithmetic
lives in ``xcf_oracle.c`` (plain C, FP64, its own FFT); this module compiles it
with gcc on first use and marshals numpy arrays through ctypes.  It shares no
code with the CUDA library.

Parity unpinned: window shape, band-pass shape and cut-offs, log-polar
sampling constants (the paper gives none of them); their implementation is
pinned to library routines (``tests/test_oracle_filters.py``), and everything
else by the tests under ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = (os.path.join(_HERE, "xcf_oracle.c"), os.path.join(_HERE, "cnn_oracle.c"))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(map(os.path.getmtime, _SRCS)):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, *_SRCS, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Opts(C.Structure):
    _fields_ = [("window", C.c_int32), ("sigma_hp", C.c_double), ("sigma_lp", C.c_double),
                ("lp_nr", C.c_int32), ("lp_neta", C.c_int32), ("lp_rmin", C.c_double),
                ("lp_rmax", C.c_double), ("upsample", C.c_int32), ("interp", C.c_int32),
                ("ndp_bg_sigma", C.c_double), ("lp_windows", C.c_int32)]


def default_opts(n: int, **kw) -> Opts:
    """Defaults: Hann window, sigma_hp = 2, sigma_lp = n/4 cycles per image,
    log-polar n/4 radii x (2n rounded up to a power of two) angles over
    r in [n/4, n/2 - 1] px in 4 radial
    windows, NDP background sigma n/8 px (0 selects it; < 0 turns the
    correction off)."""
    neta = 1
    while neta < 2 * n:   # the angular sampling is a power of two (2n for 2^k sides)
        neta *= 2
    d = dict(window=1, sigma_hp=2.0, sigma_lp=n / 4.0, lp_nr=max(n // 4, 2), lp_neta=neta,
             lp_rmin=n / 4.0, lp_rmax=n / 2.0 - 1.0, upsample=0, interp=0, ndp_bg_sigma=0.0, lp_windows=4)
    d.update(kw)
    return Opts(**d)


_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)
_I = C.POINTER(C.c_int32)


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            sig = {
                "orc_num_threads": ([], C.c_int),
                "orc_dft1": ([_D, _D, C.c_int, C.c_int], None),
                "orc_dft2_brute": ([_D, _D, C.c_int, C.c_int], None),
                "orc_fft1": ([_D, C.c_int, C.c_int], None),
                "orc_fft2": ([_D, C.c_int, C.c_int], None),
                "orc_crop": ([C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                              _I, _I, _I, _D], C.c_int),
                "orc_crop_ex": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                 _I, _I, _I, _D], C.c_int),
                "orc_bandpass": ([C.c_int, C.c_int, C.c_int, C.c_double, C.c_double], C.c_double),
                "orc_window": ([C.c_int, C.c_int, C.c_int], C.c_double),
                "orc_prep": ([_D, C.c_int, C.POINTER(Opts), _D, _D], C.c_int),
                "orc_prep_many": ([_D, C.c_int, C.c_int, C.POINTER(Opts), _D, _D, _I], None),
                "orc_xcf_surface": ([_D, _D, C.c_int, _D], None),
                "orc_xcf_spatial": ([_D, _D, C.c_int, _D], None),
                "orc_parabola": ([C.c_double, C.c_double, C.c_double], C.c_double),
                "orc_peak_upsampled": ([_D, _D, C.c_int, C.c_int, _D, _D, _D], None),
                "orc_pair_upsampled": ([_D, _D, C.c_int, C.c_int, _D, _D, _D], None),
                "orc_upsampled_value": ([_D, _D, C.c_int, C.c_double, C.c_double], C.c_double),
                "orc_peak": ([_D, C.c_int, _D, _I, _I, _D, _D], None),
                "orc_index": ([_D, C.c_int, _D, C.c_int, C.c_int, _I, _I, _D, _D, _D], None),
                "orc_pc_shift": ([_D, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, _I, _D], None),
                "orc_lambert_forward": ([_D, _D, _D], None),
                "orc_lambert_inverse": ([C.c_double, C.c_double, _D], None),
                "orc_master_lookup": ([_F, C.c_int, _D], C.c_double),
                "orc_quat_to_matrix": ([_D, _D], None),
                "orc_project": ([_F, C.c_int, _D, _D, C.c_double, C.c_double, C.c_int, _D], None),
                "orc_project_many": ([_F, C.c_int, _D, _D, C.c_int, C.c_double, C.c_double,
                                      C.c_int, _D, C.c_int], None),
                "orc_grid_interp": ([_F, C.c_int, C.c_double, C.c_double, C.c_int], C.c_double),
                "orc_qmul": ([_D, _D, _D], None),
                "orc_cubic_ops": ([_D], None),
                "orc_disorientation": ([_D, _D], C.c_double),
                "orc_disorientation_many": ([_D, _D, C.c_int, _D], None),
                "orc_logpolar": ([_D, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _D], None),
                "orc_eta_xcf": ([_D, _D, C.c_int, C.c_int, _D, _D], C.c_double),
                "orc_refine_one": ([_F, C.c_int, _D, C.c_double, C.c_double, C.POINTER(Opts), _F,
                                    C.c_int, _D, C.c_int, C.c_double, _D, _D, _I, _D], C.c_int),
                "orc_refine_many": ([_F, C.c_int, _D, C.c_double, C.c_double, C.POINTER(Opts), _F,
                                     C.c_int, C.c_int, _D, C.c_int, C.c_double, _D, _D, _I], None),
                "orc_bf16_round": ([C.c_double], C.c_double),
                "orc_screen": ([_D, C.c_int, _D, C.c_int, C.c_long, C.c_int, _D], None),
                "orc_ndp_normalise": ([_D, C.c_long, _D], C.c_int),
                "orc_ndp_background": ([_D, C.c_int, C.c_double, _D], None),
                "orc_ndp": ([_D, _D, C.c_long], C.c_double),
                "orc_ndp_index": ([_D, C.c_int, _D, C.c_int, C.c_long, _I, _D, _D], None),
                "orc_scan_orientation": ([_D, C.c_int, C.c_double, C.c_double, C.c_double, _D], None),
                "orc_rotation_scan": ([_F, C.c_int, C.c_int, _D, _D, C.c_double, C.c_double, C.POINTER(Opts),
                                       _D, C.c_int, C.c_double, _D, _D], None),
                "orc_fwhm": ([_D, C.c_int, C.c_double], C.c_double),
                "orc_eta_windows": ([_D, _D, C.c_int, C.c_int, C.c_int, _D], C.c_double),
                "orc_so3_grid": ([C.c_double, C.c_int, _D, C.c_long], C.c_long),
                "orc_nearest_disorientation": ([_D, C.c_int, _D, C.c_int, C.c_int, _D, _I], None),
                "orc_cnn_num_params": ([C.c_int], C.c_long),
                "orc_cnn_standardise": ([_D, C.c_int, _D], None),
                "orc_conv3x3s2": ([_D, C.c_int, C.c_int, _D, _D, C.c_int, _D], None),
                "orc_gram_schmidt": ([_D, _D], None),
                "orc_gram_schmidt_backward": ([_D, _D, _D], None),
                "orc_cubic_matrices": ([_D], None),
                "orc_cnn_head_loss": ([_D, C.c_int, _D, _D, _I, _I], C.c_double),
                "orc_cnn_forward": ([_F, _D, C.c_int, C.c_int, _D], None),
                "orc_cnn_forward_bf16": ([_F, _D, C.c_int, C.c_int, _D], None),
                "orc_cnn_loss_grad": ([_F, _D, C.c_int, C.c_int, _D, _D, _I], C.c_double),
                "orc_adam": ([_D, _D, _D, _D, C.c_long, C.c_int, C.c_double, C.c_double, C.c_double,
                              C.c_double], None),
                "orc_matrix_to_quat": ([_D, _D], None),
                "orc_cnn_proposals": ([_D, C.c_int, C.c_int, _D], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _f(a):
    return a.ctypes.data_as(_F)


def _i(a):
    return a.ctypes.data_as(_I)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def num_threads() -> int:
    return _lib_handle().orc_num_threads()


# ---------------------------------------------------------------- transforms
def dft1(x, sign=-1):
    x = _c128(x)
    out = np.empty_like(x)
    _lib_handle().orc_dft1(_d(x), _d(out), x.shape[0], sign)
    return out


def dft2_brute(x, sign=-1):
    x = _c128(x)
    out = np.empty_like(x)
    _lib_handle().orc_dft2_brute(_d(x), _d(out), x.shape[0], sign)
    return out


def fft1(x, sign=-1):
    x = _c128(x).copy()
    _lib_handle().orc_fft1(_d(x), x.shape[0], sign)
    return x


def fft2(x, sign=-1):
    x = _c128(x).copy()
    _lib_handle().orc_fft2(_d(x), x.shape[0], sign)
    return x


# ------------------------------------------------------------ pre-processing
def crop(W, H, pc, cap=256, native=False):
    """Centred crop (2^k sides, or with native=True also 96 and 160):
    returns (n, off_x, off_y, pc_cropped)."""
    n, ox, oy = C.c_int32(), C.c_int32(), C.c_int32()
    out = np.zeros(3)
    rc = _lib_handle().orc_crop_ex(W, H, cap, int(native), pc[0], pc[1], pc[2], C.byref(n), C.byref(ox),
                                   C.byref(oy), _d(out))
    if rc != 0:
        raise ValueError("detector too small")
    return n.value, ox.value, oy.value, out


def bandpass(u, v, n, sigma_hp, sigma_lp):
    return _lib_handle().orc_bandpass(u, v, n, sigma_hp, sigma_lp)


def window(k, n, kind=1):
    return _lib_handle().orc_window(k, n, kind)


def prep(img, opts=None):
    """One n x n image -> (full spectrum S [n, n] complex, spatial y [n, n], degenerate)."""
    img = _f64(img)
    n = img.shape[0]
    opts = opts or default_opts(n)
    S = np.empty((n, n), np.complex128)
    y = np.empty((n, n))
    deg = _lib_handle().orc_prep(_d(img), n, C.byref(opts), _d(S), _d(y))
    return S, y, bool(deg)


def prep_many(imgs, opts=None, want_spatial=False):
    imgs = _f64(imgs)
    P, n = imgs.shape[0], imgs.shape[1]
    opts = opts or default_opts(n)
    S = np.empty((P, n, n), np.complex128)
    y = np.empty((P, n, n)) if want_spatial else None
    deg = np.zeros(P, np.int32)
    _lib_handle().orc_prep_many(_d(imgs), P, n, C.byref(opts), _d(S),
                                _d(y) if y is not None else None, _i(deg))
    return S, y, deg


# --------------------------------------------------------------- correlation
def xcf_surface(St, Sp):
    St, Sp = _c128(St), _c128(Sp)
    n = St.shape[0]
    r = np.empty((n, n))
    _lib_handle().orc_xcf_surface(_d(St), _d(Sp), n, _d(r))
    return r


def xcf_spatial(a, b):
    a, b = _f64(a), _f64(b)
    n = a.shape[0]
    r = np.empty((n, n))
    _lib_handle().orc_xcf_spatial(_d(a), _d(b), n, _d(r))
    return r


def parabola(cm, c0, cp):
    return _lib_handle().orc_parabola(cm, c0, cp)


def peak(r):
    """-> (peak, (sy, sx), (dx, dy))"""
    r = _f64(r)
    n = r.shape[0]
    pk = C.c_double()
    sy, sx = C.c_int32(), C.c_int32()
    dx, dy = C.c_double(), C.c_double()
    _lib_handle().orc_peak(_d(r), n, C.byref(pk), C.byref(sy), C.byref(sx), C.byref(dx),
                           C.byref(dy))
    return pk.value, (sy.value, sx.value), (dx.value, dy.value)


def pair_upsampled(St, Sp, U):
    """Up-sampled peak of one pair (full spectra [n, n]) -> (peak, (dx, dy))."""
    St, Sp = _c128(St), _c128(Sp)
    n = St.shape[0]
    pk, dx, dy = C.c_double(), C.c_double(), C.c_double()
    _lib_handle().orc_pair_upsampled(_d(St), _d(Sp), n, int(U), C.byref(pk), C.byref(dx), C.byref(dy))
    return pk.value, (dx.value, dy.value)


def upsampled_value(St, Sp, y, x):
    St, Sp = _c128(St), _c128(Sp)
    return _lib_handle().orc_upsampled_value(_d(St), _d(Sp), St.shape[0], float(y), float(x))


def index(St, Sp, degenerate=None, want_all=False, pcs=None, geom=None):
    """Library search. St [T,n,n], Sp [P,n,n] full spectra.
    pcs [P,3] with geom = (W, H, pcx_lib, pcy_lib): per-pattern pattern
    centres; the shift is then taken relative to the template at the
    pattern's own centre (orc_pc_shift).
    -> best [P] int32, peak [P], shift [P,2] (dx, dy), peaks_all [P,T] or None."""
    St, Sp = _c128(St), _c128(Sp)
    T, n = St.shape[0], St.shape[1]
    P = Sp.shape[0]
    deg = np.zeros(P, np.int32) if degenerate is None else np.ascontiguousarray(degenerate, np.int32)
    best = np.empty(P, np.int32)
    pk = np.empty(P)
    sh = np.empty((P, 2))
    allp = np.empty((P, T)) if want_all else None
    _lib_handle().orc_index(_d(St), T, _d(Sp), P, n, _i(deg), _i(best), _d(pk), _d(sh),
                            _d(allp) if allp is not None else None)
    if pcs is not None:
        W, H, pcx, pcy = geom
        _lib_handle().orc_pc_shift(_d(_f64(pcs)), P, float(pcx), float(pcy), int(W), int(H), _i(best), _d(sh))
    return best, pk, sh, allp


# ---------------------------------------------------------------- projection
def lambert_forward(v):
    v = _f64(v)
    X, Y = C.c_double(), C.c_double()
    _lib_handle().orc_lambert_forward(_d(v), C.byref(X), C.byref(Y))
    return X.value, Y.value


def lambert_inverse(X, Y):
    v = np.empty(3)
    _lib_handle().orc_lambert_inverse(X, Y, _d(v))
    return v


def master_lookup(master, v):
    master, v = _f32(master), _f64(v)
    return _lib_handle().orc_master_lookup(_f(master), master.shape[1], _d(v))


def quat_to_matrix(q):
    q = _f64(q)
    R = np.empty(9)
    _lib_handle().orc_quat_to_matrix(_d(q), _d(R))
    return R.reshape(3, 3)


def project(master, q, pc, n, sample_tilt=70.0, detector_tilt=0.0):
    master, q, pc = _f32(master), _f64(q), _f64(pc)
    out = np.empty((n, n))
    _lib_handle().orc_project(_f(master), master.shape[1], _d(q), _d(pc), sample_tilt,
                              detector_tilt, n, _d(out))
    return out


def project_many(master, quats, pcs, n, sample_tilt=70.0, detector_tilt=0.0, interp=0):
    """interp: master lookup, 0 bilinear, 1 bicubic (Keys, a = -1/2)."""
    master, quats = _f32(master), _f64(quats)
    pcs = _f64(np.broadcast_to(np.asarray(pcs, np.float64), (quats.shape[0], 3)))
    P = quats.shape[0]
    out = np.empty((P, n, n))
    _lib_handle().orc_project_many(_f(master), master.shape[1], _d(quats), _d(pcs), P,
                                   sample_tilt, detector_tilt, n, _d(out), int(interp))
    return out


def grid_interp(grid, fx, fy, interp):
    """One hemisphere's grid [M, M] at grid coordinates (cell centres at integers)."""
    g = _f32(grid)
    return _lib_handle().orc_grid_interp(_f(g), g.shape[0], float(fx), float(fy), int(interp))


# ---------------------------------------------------------------- symmetry
def qmul(a, b):
    a, b = _f64(a), _f64(b)
    o = np.empty(4)
    _lib_handle().orc_qmul(_d(a), _d(b), _d(o))
    return o


def cubic_ops():
    o = np.empty((24, 4))
    _lib_handle().orc_cubic_ops(_d(o))
    return o


def disorientation(qa, qb):
    """Cubic disorientation in degrees; qa, qb [4] or [n, 4]."""
    qa, qb = _f64(qa), _f64(qb)
    if qa.ndim == 1:
        return _lib_handle().orc_disorientation(_d(qa), _d(qb))
    out = np.empty(qa.shape[0])
    _lib_handle().orc_disorientation_many(_d(qa), _d(qb), qa.shape[0], _d(out))
    return out


# ------------------------------------------------------------- screen (Eq. 1)
def bf16_round(x):
    return _lib_handle().orc_bf16_round(float(x))


def screen(yp, yt, bf16=True):
    """Zero-shift scores S [P, T] = yp . yt^T in FP64 of the unit-norm filtered
    images (flattened); bf16 rounds every input to BF16 first."""
    yp = _f64(np.asarray(yp).reshape(len(yp), -1))
    yt = _f64(np.asarray(yt).reshape(len(yt), -1))
    S = np.empty((yp.shape[0], yt.shape[0]))
    _lib_handle().orc_screen(_d(yp), yp.shape[0], _d(yt), yt.shape[0], yp.shape[1], 1 if bf16 else 0, _d(S))
    return S


# ------------------------------------------------- NDP and peak-width scans
def ndp_normalise(img):
    """Contrast normalisation (zero mean, unit population std) -> (out, degenerate)."""
    img = _f64(img)
    out = np.empty_like(img)
    deg = _lib_handle().orc_ndp_normalise(_d(img), img.size, _d(out))
    return out, bool(deg)


def ndp_background(img, sigma=0.0):
    """Background correction before the NDP: img minus its Gaussian blur
    (sigma px; 0 = n/8; < 0 = unchanged), edges repeated."""
    img = _f64(img)
    out = np.empty_like(img)
    _lib_handle().orc_ndp_background(_d(img), img.shape[0], float(sigma), _d(out))
    return out


def ndp(a, b):
    """Eq. 1 between two images of the same size."""
    a, b = _f64(a), _f64(b)
    assert a.size == b.size
    return _lib_handle().orc_ndp(_d(a), _d(b), a.size)


def ndp_index(pats, tmpl, want_all=False):
    """NDP dictionary indexing: pats [P, ...], tmpl [T, ...] images.
    -> best [P] int32 (-1 for a constant pattern), score [P], scores [P, T] or None."""
    pats = _f64(np.asarray(pats).reshape(len(pats), -1))
    tmpl = _f64(np.asarray(tmpl).reshape(len(tmpl), -1))
    P, T, d = pats.shape[0], tmpl.shape[0], pats.shape[1]
    best = np.empty(P, np.int32)
    score = np.empty(P)
    scores = np.empty((P, T)) if want_all else None
    _lib_handle().orc_ndp_index(_d(pats), P, _d(tmpl), T, d, _i(best), _d(score),
                                _d(scores) if scores is not None else None)
    return best, score, scores


def scan_orientation(q, axis, theta_rad, sample_tilt=70.0, detector_tilt=0.0):
    q = _f64(q)
    out = np.empty(4)
    _lib_handle().orc_scan_orientation(_d(q), int(axis), float(theta_rad), sample_tilt, detector_tilt, _d(out))
    return out


def rotation_scan(master, q, pc_ref, n, nh, step_deg, pc_test=None, opts=None, sample_tilt=70.0,
                  detector_tilt=0.0):
    """Fig. 3 / 4 rotation experiment on an n x n screen -> (ndp [3, L], xcf [3, L]), L = 2 nh + 1."""
    master, q = _f32(master), _f64(q)
    pc_ref = _f64(pc_ref)
    pc_test = pc_ref if pc_test is None else _f64(pc_test)
    o = opts or default_opts(n)
    L = 2 * nh + 1
    ndp_out, xcf_out = np.empty((3, L)), np.empty((3, L))
    _lib_handle().orc_rotation_scan(_f(master), master.shape[1], n, _d(pc_ref), _d(pc_test), sample_tilt,
                                    detector_tilt, C.byref(o), _d(q), int(nh), float(step_deg), _d(ndp_out),
                                    _d(xcf_out))
    return ndp_out, xcf_out


def fwhm(curve, step):
    """Full width at half maximum of a centred curve (units of step); -1 if unresolved."""
    c = _f64(curve)
    return _lib_handle().orc_fwhm(_d(c), c.size, float(step))


# ---------------------------------------------------------------- SO(3) sampling
def so3_grid(step_deg, dedup=True):
    """S^2 x S^1 library generator in the cubic fundamental zone -> [T, 4]."""
    lib = _lib_handle()
    n = lib.orc_so3_grid(float(step_deg), int(dedup), None, 0)
    out = np.empty((n, 4))
    lib.orc_so3_grid(float(step_deg), int(dedup), _d(out), n)
    return out


def nearest_disorientation(qa, qb=None, mode=None):
    """Nearest qb (cubic disorientation) of every qa -> (angle_deg [na], index [na]).
    qb None: qa against itself excluding self (mode 1); mode 2: earlier entries only."""
    qa = _f64(qa)
    same = qb is None
    qb = qa if same else _f64(qb)
    if mode is None:
        mode = 1 if same else 0
    ang = np.empty(len(qa))
    idx = np.empty(len(qa), np.int32)
    _lib_handle().orc_nearest_disorientation(_d(qa), len(qa), _d(qb), len(qb), int(mode), _d(ang), _i(idx))
    return ang, idx


# ---------------------------------------------------------------- refinement
def logpolar(img, opts=None):
    img = _f64(img)
    n = img.shape[0]
    o = opts or default_opts(n)
    out = np.empty((o.lp_nr, o.lp_neta))
    _lib_handle().orc_logpolar(_d(img), n, o.lp_nr, o.lp_neta, o.lp_rmin, o.lp_rmax, _d(out))
    return out


def eta_xcf(a, b):
    """-> (shift along eta in samples, peak, c [neta])"""
    a, b = _f64(a), _f64(b)
    nr, ne = a.shape
    pk = C.c_double()
    c = np.empty(ne)
    sh = _lib_handle().orc_eta_xcf(_d(a), _d(b), nr, ne, C.byref(pk), _d(c))
    return sh, pk.value, c


def eta_windows(a, b, windows):
    """Multiple-window Z measurement -> (median band shift, largest band peak)"""
    a, b = _f64(a), _f64(b)
    nr, ne = a.shape
    pk = C.c_double()
    sh = _lib_handle().orc_eta_windows(_d(a), _d(b), nr, ne, int(windows), C.byref(pk))
    return sh, pk.value


def refine_one(master, pattern, seed, pc, max_it=2, tol_deg=1e-3, opts=None,
               sample_tilt=70.0, detector_tilt=0.0):
    """-> (q [4], peak, iters, trace [iters, 4] = (dx, dy, deta, update_deg))"""
    master, pattern = _f32(master), _f32(pattern)
    n = pattern.shape[0]
    o = opts or default_opts(n)
    seed, pc = _f64(seed), _f64(pc)
    q = np.empty(4)
    pk = C.c_double()
    it = C.c_int32()
    trace = np.zeros((max(max_it, 1), 4))
    _lib_handle().orc_refine_one(_f(master), master.shape[1], _d(pc), sample_tilt, detector_tilt,
                                 C.byref(o), _f(pattern), n, _d(seed), max_it, tol_deg, _d(q),
                                 C.byref(pk), C.byref(it), _d(trace))
    return q, pk.value, it.value, trace[:it.value]


def refine_many(master, patterns, seeds, pcs, max_it=2, tol_deg=1e-3, opts=None,
                sample_tilt=70.0, detector_tilt=0.0):
    """-> (quats [P,4], peaks [P], iters [P])"""
    master, patterns = _f32(master), _f32(patterns)
    P, n = patterns.shape[0], patterns.shape[1]
    o = opts or default_opts(n)
    seeds = _f64(seeds)
    pcs = _f64(np.broadcast_to(np.asarray(pcs, np.float64), (P, 3)))
    q = np.empty((P, 4))
    pk = np.empty(P)
    it = np.empty(P, np.int32)
    _lib_handle().orc_refine_many(_f(master), master.shape[1], _d(pcs), sample_tilt,
                                  detector_tilt, C.byref(o), _f(patterns), P, n, _d(seeds),
                                  max_it, tol_deg, _d(q), _d(pk), _i(it))
    return q, pk, it


# ------------------------------------------------------- learned proposal
CNN_SIDE = 128


def cnn_num_params(k: int = 8) -> int:
    return int(_lib_handle().orc_cnn_num_params(k))


def cnn_standardise(x):
    x = _f64(x)
    y = np.empty_like(x)
    _lib_handle().orc_cnn_standardise(_d(x), x.size, _d(y))
    return y


def conv3x3s2(x, w, b=None):
    """x [Ci, s, s], w [Co, Ci, 3, 3], b [Co] -> [Co, s/2, s/2] (no activation)."""
    x, w = _f64(x), _f64(w)
    ci, s = x.shape[0], x.shape[1]
    co = w.shape[0]
    y = np.empty((co, s // 2, s // 2))
    _lib_handle().orc_conv3x3s2(_d(x), ci, s, _d(w), _d(_f64(b)) if b is not None else None, co, _d(y))
    return y


def gram_schmidt(a):
    a = _f64(a)
    R = np.empty((3, 3))
    _lib_handle().orc_gram_schmidt(_d(a), _d(R))
    return R


def gram_schmidt_backward(a, G):
    ga = np.empty(6)
    _lib_handle().orc_gram_schmidt_backward(_d(_f64(a)), _d(_f64(G)), _d(ga))
    return ga


def cubic_matrices():
    S = np.empty((24, 3, 3))
    _lib_handle().orc_cubic_matrices(_d(S))
    return S


def cnn_head_loss(out6, k, q_gt, want_grad=True):
    """-> (loss, dL/dout6 [6k] or None, head, operator)"""
    out6 = _f64(out6)
    g = np.empty(6 * k) if want_grad else None
    h, s = C.c_int32(), C.c_int32()
    loss = _lib_handle().orc_cnn_head_loss(_d(out6), k, _d(_f64(q_gt)), _d(g) if g is not None else None,
                                           C.byref(h), C.byref(s))
    return loss, g, h.value, s.value


def cnn_forward(params, x, k=8):
    """params float32 [n], x [B, 128, 128] -> out [B, 6k] (FP64)."""
    x = _f64(x)
    B = x.shape[0]
    out = np.empty((B, 6 * k))
    _lib_handle().orc_cnn_forward(_f(_f32(params)), _d(x), B, k, _d(out))
    return out


def cnn_forward_bf16(params, x, k=8):
    """The BF16 inference form: convolutions 2..5 on BF16-rounded inputs and weights."""
    x = _f64(x)
    B = x.shape[0]
    out = np.empty((B, 6 * k))
    _lib_handle().orc_cnn_forward_bf16(_f(_f32(params)), _d(x), B, k, _d(out))
    return out


def cnn_loss_grad(params, x, q_gt, k=8, want_grad=True):
    """-> (mean loss, grad [n] FP64 or None, winners [B, 2])"""
    x = _f64(x)
    B = x.shape[0]
    grad = np.empty(cnn_num_params(k)) if want_grad else None
    win = np.empty((B, 2), np.int32)
    loss = _lib_handle().orc_cnn_loss_grad(_f(_f32(params)), _d(x), B, k, _d(_f64(q_gt)),
                                           _d(grad) if grad is not None else None, _i(win))
    return loss, grad, win


def adam(params, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In place on FP64 arrays params, m, v."""
    _lib_handle().orc_adam(_d(params), _d(_f64(grad)), _d(m), _d(v), params.size, t, lr, b1, b2, eps)


def matrix_to_quat(R):
    q = np.empty(4)
    _lib_handle().orc_matrix_to_quat(_d(_f64(R)), _d(q))
    return q


def cnn_proposals(out, k=8):
    out = _f64(out)
    B = out.shape[0]
    q = np.empty((B, k, 4))
    _lib_handle().orc_cnn_proposals(_d(out), B, k, _d(q))
    return q
