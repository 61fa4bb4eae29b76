"""Pins of the oracle on native (non power of two) detector sides, 96, 160
and 200 px: the transforms against numpy's FFT (a library routine), the native
crop rule, the correlation invariants (self peak, exact integer rolls,
brute-force spatial correlation), library matching and refinement."""
import numpy as np
import pytest

import oracle as orc
import synth

PC0 = (0.5, 0.5, 0.6)


@pytest.mark.parametrize("n", [96, 160, 200])
def test_transform_is_numpys_fft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    np.testing.assert_allclose(orc.fft2(x), np.fft.fft2(x), atol=1e-9 * n * n)
    np.testing.assert_allclose(orc.fft2(x, +1), np.fft.ifft2(x) * n * n, atol=1e-9 * n * n)


def test_native_crop_sides():
    # the largest side of {16, 32, 64, 96, 128, 160, 200, 256} that fits; PC kept on the same pixel
    assert orc.crop(96, 96, PC0, native=True)[:3] == (96, 0, 0)
    assert orc.crop(160, 160, PC0, native=True)[:3] == (160, 0, 0)
    assert orc.crop(200, 200, PC0, native=True)[:3] == (200, 0, 0)
    assert orc.crop(240, 210, PC0, native=True)[:3] == (200, 20, 5)
    assert orc.crop(300, 256, PC0, native=True)[:3] == (256, 22, 0)
    n, ox, oy, pc = orc.crop(200, 180, (0.4, 0.45, 0.6), native=True)
    assert (n, ox, oy) == (160, 20, 10)
    np.testing.assert_allclose(pc, [(0.4 * 200 - 20) / 160, (0.45 * 180 - 10) / 160, 0.6 * 200 / 160])
    assert orc.crop(96, 96, PC0)[0] == 64 and orc.crop(200, 200, PC0)[0] == 128   # the 2^k rule is unchanged


@pytest.mark.parametrize("n", [96, 160, 200])
def test_self_peak_and_integer_rolls(n):
    master = synth.master_pattern("bcc", 512)
    img = orc.project_many(master, synth.random_quaternions(1, 3), PC0, n)[0]
    S, _, deg = orc.prep(img)
    assert not deg
    pk, (sy, sx), _ = orc.peak(orc.xcf_surface(S, S))
    assert pk == pytest.approx(1.0, abs=1e-12) and (sy, sx) == (0, 0)
    opts = orc.default_opts(n, window=0)
    S0, _, _ = orc.prep(img, opts)
    for dy, dx in ((3, -5), (-7, 11)):
        S1, _, _ = orc.prep(np.roll(img, (dy, dx), axis=(0, 1)), opts)
        _, (sy, sx), _ = orc.peak(orc.xcf_surface(S0, S1))
        assert (sy, sx) == (dy % n, dx % n)


def test_spatial_correlation_equals_fft_correlation_off_power_of_two():
    """Eq. 2 by brute force against Eq. 3 through the transform, 24 x 24."""
    rng = np.random.default_rng(5)
    a, b = rng.standard_normal((24, 24)), rng.standard_normal((24, 24))
    A, B = orc.fft2(a), orc.fft2(b)
    r_fft = orc.xcf_surface(A / 24, B / 24)
    np.testing.assert_allclose(r_fft, orc.xcf_spatial(a, b), atol=1e-10)


def test_library_match_and_refinement_at_96():
    master = synth.master_pattern("bcc", 512)
    n = 96
    lib = synth.random_quaternions(12, 7)
    St, _, _ = orc.prep_many(orc.project_many(master, lib, PC0, n))
    pats = orc.project_many(master, lib[[2, 9]], PC0, n)
    Sp, _, deg = orc.prep_many(pats)
    best, pk, sh, _ = orc.index(St, Sp, deg)
    assert best.tolist() == [2, 9]
    np.testing.assert_allclose(pk, 1.0, atol=1e-12)
    truth = synth.perturb(lib[:2], 2.0, 8)
    pts = orc.project_many(master, truth, PC0, n).astype(np.float32)
    q, _, it = orc.refine_many(master, pts, lib[:2], PC0, max_it=6)
    assert orc.disorientation(q, truth).max() < 0.02


def test_library_match_at_200():
    """A pattern simulated at a library orientation returns that template with
    peak 1 on the native 200 px side (lines of 200 = 8 x 25 points as direct
    DFTs)."""
    master = synth.master_pattern("bcc", 512)
    n = 200
    lib = synth.random_quaternions(6, 17)
    St, _, _ = orc.prep_many(orc.project_many(master, lib, PC0, n))
    Sp, _, deg = orc.prep_many(orc.project_many(master, lib[[4, 1]], PC0, n))
    best, pk, sh, _ = orc.index(St, Sp, deg)
    assert best.tolist() == [4, 1]
    np.testing.assert_allclose(pk, 1.0, atol=1e-12)
    np.testing.assert_allclose(sh, 0.0, atol=1e-9)
