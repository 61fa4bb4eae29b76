"""Pins of the oracle's cross-correlation, peak search and library search
(Eqs. 1-3 and 6, Fig. 1 A-C, the peak up-sampling of the FFT section)."""
import numpy as np
import pytest


def _filtered_pair(orc, n, seed, **kw):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n))
    b = rng.standard_normal((n, n))
    o = orc.default_opts(n, **kw)
    Sa, ya, _ = orc.prep(a, o)
    Sb, yb, _ = orc.prep(b, o)
    return Sa, ya, Sb, yb


def test_fft_xcf_equals_brute_spatial_xcf_16(orc):
    """Eq. 3 (FFT route) against Eq. 2 (direct sum, indices mod n)."""
    Sa, ya, Sb, yb = _filtered_pair(orc, 16, 0, sigma_lp=6.0)
    r_fft = orc.xcf_surface(Sa, Sb)
    r_dir = orc.xcf_spatial(ya, yb)
    np.testing.assert_allclose(r_fft, r_dir, atol=1e-12)


def test_zero_shift_is_normalised_dot_product(orc):
    """r(0) equals the inner product of the unit-norm filtered images (Eq. 1's NDP)."""
    Sa, ya, Sb, yb = _filtered_pair(orc, 32, 1)
    r = orc.xcf_surface(Sa, Sb)
    assert r[0, 0] == pytest.approx(float(np.sum(ya * yb)), abs=1e-13)


def test_self_correlation_and_cauchy_schwarz(orc):
    Sa, _, Sb, _ = _filtered_pair(orc, 64, 2)
    r = orc.xcf_surface(Sa, Sa)
    pk, (sy, sx), (dx, dy) = orc.peak(r)
    assert pk == pytest.approx(1.0, abs=1e-12) and (sy, sx) == (0, 0) and (dx, dy) == (0.0, 0.0)
    assert np.abs(orc.xcf_surface(Sa, Sb)).max() <= 1.0 + 1e-12


@pytest.mark.parametrize("d", [(3, -5), (0, 7), (-31, 12), (31, -32)])
def test_roll_recovers_exact_shift(orc, d):
    """Pattern = template translated by +d -> peak 1 at d (window off so that
    the whole pre-processing commutes with the translation)."""
    n = 64
    rng = np.random.default_rng(11)
    img = rng.standard_normal((n, n))
    o = orc.default_opts(n, window=0)
    St, _, _ = orc.prep(img, o)
    Sp, _, _ = orc.prep(np.roll(img, d, axis=(0, 1)), o)
    pk, (sy, sx), (dx, dy) = orc.peak(orc.xcf_surface(St, Sp))
    assert pk == pytest.approx(1.0, abs=1e-12)
    wrap = lambda s: s if s < n // 2 else s - n
    assert (sy, sx) == (d[0] % n, d[1] % n)
    assert (dy, dx) == (wrap(d[0] % n), wrap(d[1] % n))


def test_parabola(orc):
    # exact on a sampled parabola with vertex at +0.3
    f = lambda x: 2.0 - 3.0 * (x - 0.3) ** 2
    assert orc.parabola(f(-1), f(0), f(1)) == pytest.approx(0.3, abs=1e-14)
    assert orc.parabola(1.0, 1.0, 1.0) == 0.0          # flat: no fit
    assert orc.parabola(0.5, 1.0, 1.2) == 0.5          # clamped
    assert orc.parabola(0.0, 1.0, 5.0) == 0.0          # curving up: no fit


def test_subpixel_on_fourier_shifted_image(orc):
    """A band-limited image shifted by a fraction of a pixel (phase ramp):
    the parabolic fit recovers the shift to 0.05 px for a peak a few pixels
    wide, and to 0.1 px with the default (sharper) low-pass."""
    n = 64
    rng = np.random.default_rng(4)
    for slp, tol in [(n / 8, 0.05), (n / 4, 0.1)]:
        _check_subpixel(orc, n, rng, slp, tol)


def _check_subpixel(orc, n, rng, slp, tol):
    o = orc.default_opts(n, window=0, sigma_lp=slp)
    St, _, _ = orc.prep(rng.standard_normal((n, n)), o)
    f = np.fft.fftfreq(n) * n
    for (sy, sx) in [(0.3, -0.2), (-0.45, 0.1), (2.25, -3.4)]:
        ramp = np.exp(-2j * np.pi * (f[:, None] * sy + f[None, :] * sx) / n)
        Sp = St * ramp
        Sp[n // 2, :] = 0
        Sp[:, n // 2] = 0
        Sp /= np.linalg.norm(Sp)
        _, _, (dx, dy) = orc.peak(orc.xcf_surface(St, Sp))
        assert abs(dx - sx) < tol and abs(dy - sy) < tol


def test_peak_ties_lowest_row_major(orc):
    r = np.zeros((16, 16))
    r[3, 9] = r[2, 15] = r[7, 0] = 1.0
    pk, (sy, sx), _ = orc.peak(r)
    assert (sy, sx) == (2, 15)


def test_index_search_and_ties(orc):
    n = 32
    rng = np.random.default_rng(9)
    imgs = rng.standard_normal((5, n, n))
    St, _, _ = orc.prep_many(imgs)
    St = np.concatenate([St, St[2:3]])            # template 5 duplicates template 2
    pats = np.stack([np.roll(imgs[2], (1, 2), axis=(0, 1)), imgs[4], np.full((n, n), 1.0)])
    Sp, _, deg = orc.prep_many(pats, orc.default_opts(n, window=0))
    St0, _, _ = orc.prep_many(imgs, orc.default_opts(n, window=0))
    St0 = np.concatenate([St0, St0[2:3]])
    best, pk, sh, allp = orc.index(St0, Sp, deg, want_all=True)
    assert list(best) == [2, 4, -1]                 # tie 2 vs 5 -> lowest index
    assert pk[0] == pytest.approx(1.0) and pk[1] == pytest.approx(1.0) and pk[2] == 0.0
    np.testing.assert_allclose(sh[0], [2.0, 1.0], atol=1e-9)
    assert allp.shape == (3, 6) and allp[0, 2] == allp[0, 5]
    assert np.all(allp[:2] <= 1.0 + 1e-12)
    # per-template peak is the maximum of the surface
    r = orc.xcf_surface(St0[1], Sp[0])
    assert allp[0, 1] == r.max()


def test_per_pattern_pc_is_a_translation_and_is_taken_out(orc):
    """A pattern whose pattern centre differs from the library's by
    (dx, dy) in (pcx, pcy) is the library projection translated by
    (dx W, dy H) px (the gnomonic ray of each pixel moves with the centre):
    the raw search shift recovers that translation and the per-pattern
    centre correction leaves only the orientation's part, here zero."""
    import synth
    n = 64
    pc0 = np.array([0.5, 0.5, 0.6])
    master = synth.master_pattern("bcc", 512)
    lq = synth.random_quaternions(5, 71)
    St, _, _ = orc.prep_many(orc.project_many(master, lq, pc0, n))
    moves = np.array([[3, -2], [-5, 4], [0, 6]])
    pcs = np.array([pc0 + [mx / n, my / n, 0.0] for mx, my in moves])
    pats = np.stack([orc.project(master, lq[t], pcs[i], n) for i, t in enumerate([2, 4, 0])])
    # the translation itself: interior pixels equal the library projection rolled by the move
    ref = orc.project(master, lq[2], pc0, n)
    np.testing.assert_allclose(pats[0][8:-8, 8:-8], np.roll(ref, (-2, 3), axis=(0, 1))[8:-8, 8:-8], atol=1e-12)
    Sp, _, deg = orc.prep_many(pats)
    b_raw, _, sh_raw, _ = orc.index(St, Sp, deg)
    b, pk, sh, _ = orc.index(St, Sp, deg, pcs=pcs, geom=(n, n, pc0[0], pc0[1]))
    assert b.tolist() == b_raw.tolist() == [2, 4, 0]
    # the integer peak is the move exactly; the fixed window (the content moves
    # under it) and the parabola leave a sub-pixel bias of ~0.02 px per px moved
    assert np.array_equal(np.round(sh_raw), moves)
    np.testing.assert_allclose(sh_raw, moves, atol=0.2)
    np.testing.assert_allclose(sh, 0.0, atol=0.2)
    np.testing.assert_allclose(sh_raw - sh, moves, atol=1e-12)
    # the library's own centre changes nothing; degenerate patterns keep zero
    b2, _, sh2, _ = orc.index(St, Sp, deg, pcs=np.tile(pc0, (3, 1)), geom=(n, n, pc0[0], pc0[1]))
    np.testing.assert_array_equal(sh2, sh_raw)
    Sz, _, dz = orc.prep_many(np.zeros((1, n, n)))
    _, _, shz, _ = orc.index(St, Sz, dz, pcs=pcs[:1], geom=(n, n, pc0[0], pc0[1]))
    assert np.all(shz == 0.0)
