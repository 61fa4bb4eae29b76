"""Pins of the oracle's Fourier machinery and pre-processing (Eq. 4, FFT section).

Each check is against something other than the oracle itself: a brute-force
DFT, numpy.fft (a library routine, test-only), Parseval, closed-form DFTs and
the invariances the paper's contrast normalisation implies.
"""
import numpy as np
import pytest


def _rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("n", [16, 32, 64])
def test_fft1_matches_brute_dft(orc, n):
    rng = np.random.default_rng(n)
    x = _rand_c(rng, n)
    for sign in (-1, 1):
        np.testing.assert_allclose(orc.fft1(x, sign), orc.dft1(x, sign), atol=1e-10)


def test_fft2_matches_brute_dft2_16(orc):
    rng = np.random.default_rng(1)
    x = _rand_c(rng, 16, 16)
    for sign in (-1, 1):
        np.testing.assert_allclose(orc.fft2(x, sign), orc.dft2_brute(x, sign), atol=1e-10)


@pytest.mark.parametrize("n", [16, 64, 128])
def test_fft2_matches_numpy(orc, n):
    rng = np.random.default_rng(n + 7)
    x = _rand_c(rng, n, n)
    np.testing.assert_allclose(orc.fft2(x, -1), np.fft.fft2(x), atol=1e-9 * n)
    np.testing.assert_allclose(orc.fft2(x, +1), np.fft.ifft2(x) * n * n, atol=1e-9 * n)


def test_parseval_and_roundtrip(orc):
    rng = np.random.default_rng(3)
    n = 64
    x = _rand_c(rng, n, n)
    X = orc.fft2(x, -1)
    assert np.isclose(np.sum(np.abs(x) ** 2), np.sum(np.abs(X) ** 2) / n ** 2, rtol=1e-12)
    np.testing.assert_allclose(orc.fft2(X, +1) / n ** 2, x, atol=1e-12)


def test_dft_of_delta_and_constant(orc):
    n = 32
    d = np.zeros((n, n), complex)
    d[0, 0] = 1
    np.testing.assert_allclose(orc.fft2(d), np.ones((n, n)), atol=1e-13)
    c = np.ones((n, n), complex)
    X = orc.fft2(c)
    expect = np.zeros((n, n), complex)
    expect[0, 0] = n * n
    np.testing.assert_allclose(X, expect, atol=1e-9)
    # a single plane wave lands in a single bin
    u0, v0 = 3, 5
    r, cc = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    w = np.exp(2j * np.pi * (u0 * r + v0 * cc) / n)
    X = orc.fft2(w)
    assert abs(X[u0, v0] - n * n) < 1e-8
    X[u0, v0] = 0
    assert np.abs(X).max() < 1e-8


def test_crop_worked_example(orc):
    """Paper, FFT section footnote 2: 200 -> 128 px, PCx 0.4 -> 0.34."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "pc_crop.json")))
    n, ox, oy, pc = orc.crop(g["width"], g["height"], (g["pcx_before"], 0.5, 0.6), cap=g["crop_to"])
    assert n == g["crop_to"] and ox == oy == 36
    assert round(pc[0], g["printed_decimals"]) == g["pcx_after_printed"]
    assert pc[0] == pytest.approx(0.34375, abs=1e-15)
    # the pattern centre keeps pointing at the same physical pixel
    assert pc[0] * n + ox == pytest.approx(g["pcx_before"] * g["width"])
    # the detector distance in pixels is unchanged
    assert pc[2] * n == pytest.approx(0.6 * 200)
    # largest power of two, capped
    assert orc.crop(160, 120, (0.5, 0.5, 0.6), cap=256)[0] == 64
    assert orc.crop(512, 480, (0.5, 0.5, 0.6), cap=256)[0] == 256
    with pytest.raises(ValueError):
        orc.crop(15, 40, (0.5, 0.5, 0.6))


def test_filter_and_window_shapes(orc):
    n = 64
    assert orc.bandpass(0, 0, n, 2.0, 16.0) == 0.0
    for (u, v) in [(1, 2), (5, 60), (31, 33), (32, 0)]:
        assert orc.bandpass(u, v, n, 2.0, 16.0) == pytest.approx(
            orc.bandpass((n - u) % n, (n - v) % n, n, 2.0, 16.0))
    # Gaussian high-pass x low-pass at rho^2 = 25
    assert orc.bandpass(3, 4, n, 2.0, 16.0) == pytest.approx(
        (1 - np.exp(-25 / 8)) * np.exp(-25 / 512), rel=1e-14)
    assert orc.window(0, n, 1) == 0.0 and orc.window(n // 2, n, 1) == pytest.approx(1.0)
    assert orc.window(5, n, 0) == 1.0


def test_prep_normalisation_and_invariances(orc):
    rng = np.random.default_rng(5)
    n = 64
    img = rng.standard_normal((n, n)) * 3 + 10
    S, y, deg = orc.prep(img)
    assert not deg
    assert np.sum(np.abs(S) ** 2) == pytest.approx(1.0, abs=1e-12)
    assert np.sum(y ** 2) == pytest.approx(1.0, abs=1e-12)
    # Hermitian: the image is real
    Sm = np.conj(S[(-np.arange(n)) % n][:, (-np.arange(n)) % n])
    np.testing.assert_allclose(S, Sm, atol=1e-14)
    # y is the unitary inverse transform of S
    np.testing.assert_allclose(np.fft.fft2(y) / n, S, atol=1e-12)
    # contrast normalisation: invariant to a x + b with a > 0
    S2, _, _ = orc.prep(img * 7.5 - 3.0)
    np.testing.assert_allclose(S2, S, atol=1e-12)
    # and the spectrum is the filtered, windowed DFT of the standardised image
    o = orc.default_opts(n)
    z = (img - img.mean()) / img.std()
    h = np.array([orc.window(k, n, 1) for k in range(n)])
    z = z * h[:, None] * h[None, :]
    Hf = np.array([[orc.bandpass(u, v, n, o.sigma_hp, o.sigma_lp) for v in range(n)] for u in range(n)])
    X = np.fft.fft2(z) / n * Hf
    np.testing.assert_allclose(S, X / np.linalg.norm(X), atol=1e-12)


def test_prep_degenerate(orc):
    S, y, deg = orc.prep(np.full((32, 32), 4.0))
    assert deg and not S.any() and not y.any()
