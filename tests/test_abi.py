"""The C-ABI library loads and exports every entry point the header declares
(no GPU needed); host-only entry points behave as documented."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ebsdxcf.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(xcf_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1807_11313_gb300 import build
    return ctypes.CDLL(build.build())


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_1807_11313_gb300 import xcf
    assert sorted(xcf.exported_symbols()) == _declared()


def test_strerror_and_defaults():
    from paper_1807_11313_gb300 import xcf
    L = xcf.load()
    assert L.xcf_strerror(0) == b"ok"
    assert L.xcf_strerror(-2) == b"unsupported detector size"
    o = xcf.xcf_options()
    assert L.xcf_options_default(ctypes.byref(o)) == 0
    assert o.window == 1 and o.sigma_hp == 2.0 and o.max_iter == 2 and o.tol_deg == 1e-3


def test_crop_matches_paper_example():
    """Paper, FFT section footnote 2: 200 -> 128 px moves PCx 0.4 -> 0.34."""
    from paper_1807_11313_gb300 import xcf
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "pc_crop.json")))
    n, ox, oy, pc = xcf.xcf_crop(xcf.geometry(g["width"], g["height"], (g["pcx_before"], 0.5, 0.6)))
    assert n == g["crop_to"] and ox == 36 and oy == 36
    assert round(pc[0], 2) == g["pcx_after_printed"]
    with pytest.raises(xcf.XcfError) as e:
        xcf.xcf_crop(xcf.geometry(12, 40))
    assert e.value.code == xcf.XCF_ERR_SIZE
    # larger detectors are capped at 256
    assert xcf.xcf_crop(xcf.geometry(1200, 1000))[0] == 256


def test_native_crop_rule_matches_oracle(orc):
    """The native rule (options.native_sizes = 1) picks the same side, offsets and
    pattern centre as the oracle's; the 2^k rule stays the default."""
    from paper_1807_11313_gb300 import xcf
    for W, H, pc in ((96, 96, (0.5, 0.5, 0.6)), (200, 180, (0.4, 0.45, 0.6)), (170, 300, (0.52, 0.3, 0.7)),
                     (100, 98, (0.5, 0.5, 0.6)), (1200, 1000, (0.5, 0.5, 0.6)), (200, 200, (0.5, 0.5, 0.6)),
                     (240, 210, (0.45, 0.5, 0.62))):
        g = xcf.geometry(W, H, pc)
        n, ox, oy, pcc = xcf.xcf_crop(g, native=True)
        on, oox, ooy, opc = orc.crop(W, H, pc, native=True)
        assert (n, ox, oy) == (on, oox, ooy)
        np.testing.assert_allclose(pcc, opc, rtol=1e-15)
        assert xcf.xcf_crop(g)[:3] == orc.crop(W, H, pc)[:3]
    assert xcf.xcf_crop(xcf.geometry(96, 96), native=True)[0] == 96
    assert xcf.xcf_crop(xcf.geometry(200, 200), native=True)[0] == 200
    assert xcf.xcf_crop(xcf.geometry(96, 96))[0] == 64
    assert xcf.load().xcf_crop_ex(ctypes.byref(xcf.geometry(96, 96)), 2, None, None, None, None) == xcf.XCF_ERR_ARG


def test_noalloc_limits_cover_every_side():
    """Host-only: the fixed no-alloc scratch holds this many patterns per side
    (spectra + flags + keys in 16 MiB, each slice 256-byte aligned)."""
    from paper_1807_11313_gb300 import xcf
    def fits(n):
        H = n * (n // 2 + 1)
        r = lambda x: (x + 255) & ~255
        P = 0
        while r(8 * H * (P + 1)) + r(4 * (P + 1)) + r(8 * (P + 1)) <= 16 << 20:
            P += 1
        return P
    for n in (16, 32, 64, 96, 128, 160, 256):
        assert xcf.xcf_noalloc_max_patterns(n) == fits(n) > 0
    for n in (0, 8, 100, 200, 512):
        assert xcf.xcf_noalloc_max_patterns(n) == 0
    m = re.search(r"#define XCF_NOALLOC_SCRATCH_BYTES \((\d+)u << (\d+)\)", open(HEADER).read())
    assert xcf.XCF_NOALLOC_SCRATCH_BYTES == int(m.group(1)) << int(m.group(2)) == 16 << 20


def test_binding_checks_sizes_before_calling_c():
    """Host-only: a tensor whose element count does not match P and the
    library's detector raises ValueError before any call into the library."""
    import torch
    from paper_1807_11313_gb300 import xcf

    class _Lib:
        geom = xcf.geometry(64, 48)
        T = 7
    lib = _Lib()
    xcf._sizes(lib, 3, patterns=torch.empty(3, 48, 64), best=torch.empty(3), shift=torch.empty(3, 2),
               pcs=torch.empty(3, 3), peaks=torch.empty(3, 7))
    for bad in (dict(patterns=torch.empty(3, 64, 64)), dict(best=torch.empty(2)), dict(shift=torch.empty(3)),
                dict(pcs=torch.empty(3, 2)), dict(quats=torch.empty(3, 3)), dict(peaks=torch.empty(3, 6))):
        with pytest.raises(ValueError):
            xcf._sizes(lib, 3, **bad)


def test_network_parameter_count_matches_oracle(orc):
    """Host-only: the flat parameter count of the proposal network equals the
    oracle's layer-by-layer count, for every valid head count."""
    from paper_1807_11313_gb300 import xcf
    L = xcf.load()
    for k in (1, 2, 8, 17, 64):
        assert L.xcf_net_num_params(k) == orc.cnn_num_params(k)
    assert L.xcf_net_num_params(0) == -1 and L.xcf_net_num_params(65) == -1


def test_option_defaults_are_the_documented_readings():
    from paper_1807_11313_gb300 import xcf
    o = xcf.xcf_options()
    assert xcf.load().xcf_options_default(ctypes.byref(o)) == 0
    assert (o.window, o.sigma_hp, o.max_iter, o.tol_deg) == (1, 2.0, 2, 1e-3)
    assert o.sigma_lp == 0.0 and o.lp_nr == 0 and o.lp_neta == 0          # 0: N/4, N/4 radii, 2N angles
    assert (o.upsample, o.master_interp, o.lp_windows, o.native_sizes) == (0, 0, 0, 0)
    assert o.ndp_bg_sigma == 0.0                                          # 0: N/8 px
