"""Pins of the oracle's pre-processing filters and log-polar resampler against
library routines.  The paper names a window, a band-pass and a log-polar
transform without their constants (the readings: periodic Hann; Gaussian
high-pass x Gaussian low-pass in cycles per image; bilinear samples on
log-spaced radii about the screen centre); these tests pin the oracle's
implementation of those readings, so that a dropped factor, a wrong sign or a
transposed index in it fails."""
import numpy as np
import pytest

import oracle as orc

scipy_signal = pytest.importorskip("scipy.signal")
ndimage = pytest.importorskip("scipy.ndimage")


@pytest.mark.parametrize("n", [16, 64, 96, 128, 160])
def test_window_is_scipys_periodic_hann(n):
    w = np.array([orc.window(k, n, 1) for k in range(n)])
    np.testing.assert_allclose(w, scipy_signal.windows.hann(n, sym=False), atol=1e-15)
    assert all(orc.window(k, n, 0) == 1.0 for k in range(n))


@pytest.mark.parametrize("n,s_hp,s_lp", [(64, 2.0, 16.0), (96, 2.0, 24.0), (128, 3.0, 10.0), (32, 1.0, 8.0)])
def test_bandpass_is_a_product_of_fourier_gaussians(n, s_hp, s_lp):
    """Gaussian of sigma s (cycles per image) in frequency = scipy's
    fourier_gaussian with a spatial sigma of n / (2 pi s)."""
    H = np.array([[orc.bandpass(u, v, n, s_hp, s_lp) for v in range(n)] for u in range(n)])
    one = np.ones((n, n))
    lp = ndimage.fourier_gaussian(one, sigma=n / (2 * np.pi * s_lp))
    hp = 1.0 - ndimage.fourier_gaussian(one, sigma=n / (2 * np.pi * s_hp))
    np.testing.assert_allclose(H, hp * lp, atol=1e-14)
    assert H[0, 0] == 0.0                       # no DC
    np.testing.assert_allclose(H, H.T, atol=0)  # radial: symmetric in u, v
    np.testing.assert_allclose(H[1:, 1:], H[1:, 1:][::-1, ::-1], atol=0)   # even in the signed frequency


@pytest.mark.parametrize("n", [32, 96, 128])
def test_prep_is_the_library_composition(n):
    """Spectrum of the oracle's pre-processing = numpy's unitary FFT of the
    standardised, Hann-windowed image times the band-pass, over its norm."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n)) * 4 + 9
    opts = orc.default_opts(n)
    S, y, deg = orc.prep(x, opts)
    assert not deg
    h = scipy_signal.windows.hann(n, sym=False)
    z = (x - x.mean()) / x.std() * np.outer(h, h)
    one = np.ones((n, n))
    H = (1 - ndimage.fourier_gaussian(one, n / (2 * np.pi * opts.sigma_hp))) * \
        ndimage.fourier_gaussian(one, n / (2 * np.pi * opts.sigma_lp))
    F = np.fft.fft2(z) / n * H
    F /= np.linalg.norm(F)
    np.testing.assert_allclose(S, F, atol=1e-12)
    np.testing.assert_allclose(y, np.real(np.fft.ifft2(F)) * n, atol=1e-12)


@pytest.mark.parametrize("n", [64, 96, 128])
def test_logpolar_is_bilinear_sampling(n):
    rng = np.random.default_rng(n + 1)
    img = rng.standard_normal((n, n))
    o = orc.default_opts(n)
    lp = orc.logpolar(img, o)
    m = np.arange(o.lp_nr)
    r = o.lp_rmin * (o.lp_rmax / o.lp_rmin) ** (m / (o.lp_nr - 1))
    eta = 2 * np.pi * np.arange(o.lp_neta) / o.lp_neta
    c = n / 2 - 0.5
    rows = c - r[:, None] * np.sin(eta)[None, :]
    cols = c + r[:, None] * np.cos(eta)[None, :]
    ref = ndimage.map_coordinates(img, [rows.ravel(), cols.ravel()], order=1).reshape(lp.shape)
    np.testing.assert_allclose(lp, ref, atol=1e-12)


@pytest.mark.parametrize("n", [64, 96])
def test_logpolar_turns_a_quarter_rotation_into_a_quarter_shift(n):
    """Rotating the image a quarter turn counter-clockwise (y up) about the
    screen centre shifts the log-polar image by n_eta / 4 along eta."""
    rng = np.random.default_rng(n + 2)
    img = rng.standard_normal((n, n))
    o = orc.default_opts(n)
    a = orc.logpolar(img, o)
    b = orc.logpolar(np.rot90(img), o)
    np.testing.assert_allclose(b, np.roll(a, o.lp_neta // 4, axis=1), atol=1e-9)
