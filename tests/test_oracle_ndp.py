"""Pins of the oracle's normalised dot product (Eq. 1), its dictionary
indexing, the rotation experiment of the sampling-frequency section (Fig. 3,
Fig. 4 A-C) and the FWHM measurement, against closed forms, a library routine
(numpy's Pearson coefficient), image geometry done by scipy, and the paper's
qualitative statements."""
import math

import numpy as np
import pytest

import oracle as orc
import synth

FWHM_GAUSS = 2.0 * math.sqrt(2.0 * math.log(2.0))   # FWHM / sigma of a Gaussian


# ------------------------------------------------------------------ Eq. 1
def test_ndp_identical_negated_and_affine():
    rng = np.random.default_rng(0)
    a = rng.random((16, 16))
    assert orc.ndp(a, a) == pytest.approx(1.0, abs=1e-14)
    assert orc.ndp(a, -a) == pytest.approx(-1.0, abs=1e-14)
    # contrast normalisation makes the NDP blind to gain and offset
    assert orc.ndp(3.0 * a + 7.0, a) == pytest.approx(1.0, abs=1e-13)
    assert orc.ndp(a, -2.0 * a + 1.0) == pytest.approx(-1.0, abs=1e-13)


def test_ndp_is_pearson_coefficient():
    rng = np.random.default_rng(1)
    for _ in range(5):
        a, b = rng.normal(size=300), rng.normal(size=300) + 0.3 * np.arange(300) / 300
        assert orc.ndp(a, b) == pytest.approx(np.corrcoef(a, b)[0, 1], abs=1e-13)


def test_ndp_orthogonal_and_constant():
    assert orc.ndp(np.array([1.0, -1, 1, -1]), np.array([1.0, 1, -1, -1])) == pytest.approx(0.0, abs=1e-15)
    c = np.full((8, 8), 0.1)
    out, deg = orc.ndp_normalise(c)
    assert deg and not out.any()
    assert orc.ndp(c, np.random.default_rng(2).random((8, 8))) == 0.0


def test_ndp_normalise_moments():
    x = np.random.default_rng(3).random((32, 32)) * 50 + 3
    v, deg = orc.ndp_normalise(x)
    assert not deg
    assert v.mean() == pytest.approx(0.0, abs=1e-13)
    assert v.std() == pytest.approx(1.0, abs=1e-13)   # population std


def test_ndp_index_brute_force():
    rng = np.random.default_rng(4)
    T, P = 9, 6
    tmpl = rng.random((T, 16, 16))
    tmpl[7] = tmpl[2]                  # an exact duplicate: the lower index wins
    pats = rng.random((P, 16, 16))
    pats[0] = tmpl[2] + 0.01 * rng.random((16, 16))
    pats[5] = 2.5                      # constant pattern
    best, score, allsc = orc.ndp_index(pats, tmpl, want_all=True)
    for p in range(P):
        if p == 5:
            assert best[p] == -1 and score[p] == 0.0
            continue
        ref = np.array([np.corrcoef(pats[p].ravel(), tmpl[t].ravel())[0, 1] for t in range(T)])
        np.testing.assert_allclose(allsc[p], ref, atol=1e-12)
        assert score[p] == pytest.approx(ref.max(), abs=1e-12)
        assert ref[best[p]] >= ref.max() - 1e-12
    assert best[0] == 2


# ------------------------------------------------------------------ FWHM
def test_fwhm_triangle_exact():
    step = 0.5
    th = (np.arange(81) - 40) * step
    for bl, br in ((4.0, 4.0), (3.0, 7.5), (6.25, 2.0)):
        c = np.where(th <= 0, np.clip(1 + th / bl, 0, None), np.clip(1 - th / br, 0, None))
        assert orc.fwhm(c, step) == pytest.approx(0.5 * (bl + br), abs=1e-12)


def test_fwhm_gaussian_and_baseline_free_definition():
    step = 0.05
    th = (np.arange(801) - 400) * step
    for s in (0.8, 2.0, 5.0):
        g = np.exp(-th ** 2 / (2 * s * s))
        assert orc.fwhm(g, step) == pytest.approx(FWHM_GAUSS * s, rel=2e-4)
    # half of the maximum over zero correlation: on a baseline of 0.2 the half
    # level 0.5 is the level 0.375 of the unit Gaussian on top of it
    g = 0.2 + 0.8 * np.exp(-th ** 2 / (2 * 2.0 ** 2))
    expect = 2 * 2.0 * math.sqrt(2 * math.log(1 / 0.375))
    assert orc.fwhm(g, step) == pytest.approx(expect, rel=2e-4)


def test_fwhm_unresolved_and_plateau():
    th = np.arange(21) - 10.0
    assert orc.fwhm(np.exp(-th ** 2 / 2000.0), 1.0) == -1.0      # never falls to half within the scan
    c = np.exp(-th ** 2 / 8.0)
    c[:3] = 0.9                                                   # one side climbs back above half
    assert orc.fwhm(c, 1.0) > 0
    c2 = c.copy()
    c2[:12] = 1.0                                                 # left side never falls below half
    assert orc.fwhm(c2, 1.0) == -1.0
    assert orc.fwhm(-np.ones(5), 1.0) == -1.0
    p = np.zeros(21)
    p[8:13] = 1.0                                                 # plateau of five samples, walls of one step
    assert orc.fwhm(p, 1.0) == pytest.approx(5.0, abs=1e-12)


# ------------------------------------------------------ rotation experiment
@pytest.fixture(scope="module")
def master():
    return synth.master_pattern("bcc", 1024)


def test_scan_orientation_group_properties():
    q = synth.random_quaternions(1, 11)[0]
    for ax in range(3):
        q0 = orc.scan_orientation(q, ax, 0.0)
        assert abs(abs(np.dot(q0, q)) - 1) < 1e-14
        a = orc.scan_orientation(orc.scan_orientation(q, ax, 0.3), ax, -0.1)
        b = orc.scan_orientation(q, ax, 0.2)
        assert abs(abs(np.dot(a, b)) - 1) < 1e-13
        # a rotation by theta moves the orientation by theta
        d = orc.disorientation(q, orc.scan_orientation(q, ax, math.radians(3.0)))
        assert d == pytest.approx(3.0, abs=1e-9)


def _masked_ndp(a, b, mask):
    return orc.ndp(a[mask], b[mask])


def test_scan_z_is_in_plane_rotation_about_pc(master):
    """A rotation about the detector normal rotates the pattern in the screen
    plane about the pattern centre (scipy rotates about the array centre,
    which is the PC here); rotations about x and y do not."""
    from scipy import ndimage
    n, pc = 128, (0.5, 0.5, 0.6)
    q = synth.random_quaternions(1, 3)[0]
    ref = orc.project_many(master, q[None], pc, n)[0]
    yy, xx = np.mgrid[:n, :n]
    disc = (yy - (n - 1) / 2) ** 2 + (xx - (n - 1) / 2) ** 2 < (n / 3) ** 2
    rot = ndimage.rotate(ref, 5.0, reshape=False, order=1)
    got = []
    for ax in range(3):
        t = orc.project_many(master, orc.scan_orientation(q, ax, math.radians(5.0))[None], pc, n)[0]
        got.append(_masked_ndp(t, rot, disc))
    assert got[2] > 0.995 and max(got[0], got[1]) < 0.6, got


def test_scan_x_y_are_screen_shifts(master):
    """Small rotations about detector x (y) translate the pattern near the PC
    vertically (horizontally) by pcz n tan(theta) pixels (Eq. 7)."""
    n, pc = 128, (0.5, 0.5, 0.6)
    q = synth.random_quaternions(1, 3)[0]
    ref = orc.project_many(master, q[None], pc, n)[0]
    inner = np.zeros((n, n), bool)
    inner[16:-16, 16:-16] = True
    expect = round(pc[2] * n * math.tan(math.radians(2.0)))     # 2.68 -> 3 px
    for ax, want in ((0, (expect, 0)), (1, (0, expect))):
        t = orc.project_many(master, orc.scan_orientation(q, ax, math.radians(2.0))[None], pc, n)[0]
        scores = {(sr, sc): _masked_ndp(t, np.roll(ref, (sr, sc), axis=(0, 1)), inner)
                  for sr in range(-5, 6) for sc in range(-5, 6)}
        assert max(scores, key=scores.get) == want


def test_scan_self_match_at_zero(master):
    q = synth.random_quaternions(1, 5)[0]
    nd, xc = orc.rotation_scan(master, q, (0.5, 0.3, 0.6), 64, 4, 1.0)
    np.testing.assert_allclose(nd[:, 4], 1.0, atol=1e-12)
    np.testing.assert_allclose(xc[:, 4], 1.0, atol=1e-12)
    assert np.all(nd <= 1 + 1e-12) and np.all(xc <= 1 + 1e-12)


def test_scan_matches_its_definition(master):
    """Each curve entry is Eq. 1 of the background-corrected projections / the
    FFT peak of the two projections."""
    q = synth.random_quaternions(1, 6)[0]
    n, pc, pt = 64, (0.5, 0.3, 0.6), (0.51, 0.3, 0.6)
    nd, xc = orc.rotation_scan(master, q, pc, n, 3, 2.0, pc_test=pt)
    ref = orc.project_many(master, q[None], pc, n)[0]
    Sr, _, _ = orc.prep(ref)
    for ax, j in ((0, 0), (1, 5), (2, 6)):
        qt = orc.scan_orientation(q, ax, math.radians((j - 3) * 2.0))
        t = orc.project_many(master, qt[None], pt, n)[0]
        assert nd[ax, j] == pytest.approx(orc.ndp(orc.ndp_background(ref), orc.ndp_background(t)), abs=1e-14)
        St, _, _ = orc.prep(t)
        assert xc[ax, j] == pytest.approx(orc.peak(orc.xcf_surface(Sr, St))[0], abs=1e-14)


def test_paper_claims_fft_peak_wider_than_ndp(master):
    """The FFT correlation peak is wider than the NDP peak about every axis,
    and the NDP peak is narrowest about x or y (sampling-frequency section)."""
    for seed in (5, 6, 7):
        q = synth.random_quaternions(1, seed)[0]
        nd, xc = orc.rotation_scan(master, q, (0.5, 0.3, 0.6), 128, 90, 0.5)
        wn = [orc.fwhm(nd[a], 0.5) for a in range(3)]
        wx = [orc.fwhm(xc[a], 0.5) for a in range(3)]
        assert all(w > 0 for w in wn), wn
        for a in range(3):
            assert wx[a] == -1.0 or wx[a] > wn[a], (seed, wn, wx)
        assert min(wn[0], wn[1]) < wn[2], wn


def test_pc_error_costs_ndp_more_than_fft(master):
    """A PC error translates the pattern; the FFT correlation absorbs it
    (Fig. 4 A-C: the FFT is the more tolerant method)."""
    q = synth.random_quaternions(1, 3)[0]
    pc = (0.5, 0.3, 0.6)
    for d in ((0.02, 0, 0), (0, 0.02, 0), (0, 0, 0.02)):
        nd, xc = orc.rotation_scan(master, q, pc, 128, 1, 0.5, pc_test=tuple(np.add(pc, d)))
        assert xc[0, 1] > 0.98 and nd[0, 1] < xc[0, 1] - 0.02, (d, nd[0, 1], xc[0, 1])


# ------------------------------------------------- background correction
def test_background_is_image_minus_scipy_gaussian():
    from scipy import ndimage
    rng = np.random.default_rng(8)
    for n, sigma in ((16, 1.3), (32, 0.0), (64, 5.0), (64, 11.7)):
        img = rng.random((n, n)) + np.linspace(0, 3, n)[None, :]
        s = n / 8.0 if sigma == 0 else sigma
        ref = img - ndimage.gaussian_filter(img, s, mode="nearest", truncate=3.0)
        np.testing.assert_allclose(orc.ndp_background(img, sigma), ref, atol=1e-12)


def test_background_off_constant_and_ramp():
    rng = np.random.default_rng(9)
    img = rng.random((32, 32))
    np.testing.assert_array_equal(orc.ndp_background(img, -1.0), img)
    assert np.abs(orc.ndp_background(np.full((32, 32), 4.2), 3.0)).max() < 1e-13
    # a linear ramp is reproduced by a symmetric blur away from the edges
    ramp = np.tile(np.arange(64, dtype=float), (64, 1))
    out = orc.ndp_background(ramp, 4.0)
    assert np.abs(out[:, 13:-13]).max() < 1e-12 and np.abs(out[:, :3]).max() > 0.1


def test_scan_uses_background_corrected_ndp(master):
    """The NDP curve of the scan is Eq. 1 of the background-corrected images."""
    q = synth.random_quaternions(1, 12)[0]
    n, pc = 64, (0.5, 0.3, 0.6)
    nd, _ = orc.rotation_scan(master, q, pc, n, 2, 3.0)
    nd_off, _ = orc.rotation_scan(master, q, pc, n, 2, 3.0, opts=orc.default_opts(n, ndp_bg_sigma=-1.0))
    ref = orc.project_many(master, q[None], pc, n)[0]
    t = orc.project_many(master, orc.scan_orientation(q, 1, math.radians(3.0))[None], pc, n)[0]
    assert nd[1, 3] == pytest.approx(orc.ndp(orc.ndp_background(ref), orc.ndp_background(t)), abs=1e-14)
    assert nd_off[1, 3] == pytest.approx(orc.ndp(ref, t), abs=1e-14)
