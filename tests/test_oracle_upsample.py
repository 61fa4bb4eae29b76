"""Pins of the oracle's up-sampled correlation peak (the paper's sub-pixel
"up-sampling", evaluated by the Fourier series of the correlation): equal to
the FFT surface at integer shifts, exact recovery of band-limited sub-pixel
translations to the grid step, and never below the integer peak."""
import numpy as np
import pytest


def _spectrum(n, seed, band=None):
    """Unit-norm spectrum of a real random image, zero at |f| >= band (band-limited)."""
    rng = np.random.default_rng(seed)
    S = np.fft.fft2(rng.normal(size=(n, n)))
    f = np.fft.fftfreq(n) * n
    if band is not None:
        S[(np.abs(f)[:, None] >= band) | (np.abs(f)[None, :] >= band)] = 0
    return S / np.linalg.norm(S)


def _translate(S, dy, dx):
    """Spectrum of the image translated by +(dy, dx) (rows, columns)."""
    n = S.shape[0]
    f = np.fft.fftfreq(n) * n
    return S * np.exp(-2j * np.pi * (f[:, None] * dy + f[None, :] * dx) / n)


def test_equals_fft_surface_at_integer_shifts(orc):
    n = 16
    St, Sp = _spectrum(n, 1), _spectrum(n, 2)
    r = orc.xcf_surface(St, Sp)
    for y, x in [(0, 0), (3, 5), (15, 1), (8, 8), (-2, -7)]:
        assert abs(orc.upsampled_value(St, Sp, y, x) - r[y % n, x % n]) < 1e-12


@pytest.mark.parametrize("dy,dx,U", [(0.37, -0.21, 20), (-1.44, 2.03, 25), (0.0, 0.5, 10), (3.26, -0.78, 50)])
def test_recovers_band_limited_translation(orc, dy, dx, U):
    n = 32
    St = _spectrum(n, 3, band=12)
    Sp = _translate(St, dy, dx)
    peak, (sx, sy) = orc.pair_upsampled(St, Sp, U)
    assert abs(sx - dx) <= 0.5 / U + 1e-9 and abs(sy - dy) <= 0.5 / U + 1e-9, (sx, sy)
    assert abs(peak - 1.0) < 0.02


def test_finer_than_the_parabola(orc):
    """On a band-limited translation the up-sampled estimate beats the
    3-point parabola (the default reading)."""
    n = 32
    St = _spectrum(n, 4, band=10)
    errs_up, errs_par = [], []
    for dy, dx in [(0.31, 0.12), (-0.27, 0.44), (0.45, -0.38)]:
        Sp = _translate(St, dy, dx)
        _, (ux, uy) = orc.pair_upsampled(St, Sp, 40)
        _, _, (px_, py_) = orc.peak(orc.xcf_surface(St, Sp))
        errs_up.append(max(abs(ux - dx), abs(uy - dy)))
        errs_par.append(max(abs(px_ - dx), abs(py_ - dy)))
    assert max(errs_up) <= 0.0125 + 1e-9
    assert max(errs_up) < max(errs_par)


def test_not_below_the_integer_peak(orc):
    n = 16
    St, Sp = _spectrum(n, 5), _spectrum(n, 6)
    r = orc.xcf_surface(St, Sp)
    peak, _ = orc.pair_upsampled(St, Sp, 8)
    assert peak >= r.max() - 1e-12
