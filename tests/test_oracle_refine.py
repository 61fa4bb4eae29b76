"""Pins of the oracle's log-polar step, library search on simulated patterns
and orientation refinement (Orientation and Pattern Centre Refinement section,
Eq. 7, Figs. 6-8)."""
import math

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def master():
    return synth.master_pattern("bcc", 1024)


def test_eta_xcf_recovers_roll(orc):
    rng = np.random.default_rng(0)
    a = rng.standard_normal((16, 64))
    for D in (0, 5, -9, 31):
        b = np.roll(a, D, axis=1)
        sh, pk, _ = orc.eta_xcf(a, b)
        assert pk == pytest.approx(1.0) and sh == pytest.approx(D if D >= -32 else D + 64)


def test_eta_windows_median_of_band_shifts(orc):
    """Multiple windows: radial bands correlated on their own, the median
    band shift (mean of the middle two for an even count)."""
    rng = np.random.default_rng(1)
    a = rng.standard_normal((16, 64))
    # one window is the whole-image correlation
    b = np.roll(a, 7, axis=1)
    assert orc.eta_windows(a, b, 1)[0] == pytest.approx(orc.eta_xcf(a, b)[0])
    # a common roll is recovered by every band
    for W in (2, 3, 4, 16):
        assert orc.eta_windows(a, b, W)[0] == pytest.approx(7.0)
    # one corrupted band of three is outvoted
    c = b.copy()
    c[5:10] = rng.standard_normal((5, 64))
    assert orc.eta_windows(a, c, 3)[0] == pytest.approx(7.0)
    # bands rolled by 2, 4, 6, 8 (four radii each): median (4 + 6) / 2
    d = np.concatenate([np.roll(a[4 * k:4 * k + 4], 2 * (k + 1), axis=1) for k in range(4)])
    assert orc.eta_windows(a, d, 4)[0] == pytest.approx(5.0)
    # three bands of 16 // 3 = 5, 5, 6 radii: rolls 1, 9, 3 -> median 3
    bounds = [(0, 5), (5, 10), (10, 16)]
    e = np.concatenate([np.roll(a[m0:m1], r, axis=1) for (m0, m1), r in zip(bounds, (1, 9, 3))])
    assert orc.eta_windows(a, e, 3)[0] == pytest.approx(3.0)


def test_logpolar_turns_rotation_into_eta_shift(orc):
    """Rotating an image counter-clockwise (y up) about the screen centre
    shifts its log-polar transform along eta by theta neta / 2 pi."""
    n = 64
    yy, xx = np.meshgrid(np.arange(n) - (n / 2 - 0.5), np.arange(n) - (n / 2 - 0.5), indexing="ij")
    def img_at(theta):
        # a smooth anisotropic pattern written as a function of angle and radius
        x, y = xx, -yy
        ang = np.arctan2(y, x) - theta
        r = np.hypot(x, y)
        return np.cos(3 * ang) * np.exp(-((r - 14) / 8) ** 2) + 0.5 * np.sin(ang) * np.exp(-((r - 22) / 5) ** 2)
    o = orc.default_opts(n)
    a = orc.logpolar(img_at(0.0), o)
    for theta in (math.radians(4.0), math.radians(-7.5)):
        b = orc.logpolar(img_at(theta), o)
        sh, _, _ = orc.eta_xcf(a, b)
        assert sh == pytest.approx(theta * o.lp_neta / (2 * math.pi), abs=0.15)


def test_search_returns_library_orientation(orc, master):
    """A noise-free pattern simulated at library orientation t returns t with
    peak ~1 and zero shift (Fig. 1 B-C)."""
    n = 64
    lib = synth.random_quaternions(40, 21)
    pc = (0.5, 0.5, 0.6)
    St, _, _ = orc.prep_many(orc.project_many(master, lib, pc, n))
    pick = [3, 17, 39]
    Sp, _, deg = orc.prep_many(orc.project_many(master, lib[pick], pc, n))
    best, pk, sh, _ = orc.index(St, Sp, deg)
    assert list(best) == pick
    assert np.all(pk > 0.999999)
    assert np.abs(sh).max() < 1e-6


def test_search_tolerates_pc_shift(orc, master):
    """A pattern-centre offset becomes a translation that the XCF absorbs
    (point 2 of the introduction): the right template still wins."""
    n = 64
    lib = synth.random_quaternions(30, 22)
    St, _, _ = orc.prep_many(orc.project_many(master, lib, (0.5, 0.5, 0.6), n))
    Sp, _, deg = orc.prep_many(orc.project_many(master, lib[[4, 9]], (0.53, 0.47, 0.6), n))
    best, pk, sh, _ = orc.index(St, Sp, deg)
    assert list(best) == [4, 9]
    # shift of the PC by (+0.03 n, -0.03 n) moves the pattern right and up
    assert sh[:, 0].mean() > 1.0 and sh[:, 1].mean() < -1.0


def test_refine_recovers_perturbation(orc, master):
    """g_lib composed with a rotation of up to 5 deg per axis is recovered to
    0.01 deg noise-free; the update converges within a few iterations."""
    n = 128
    pc = np.array([0.5, 0.5, 0.6])
    ql = synth.random_quaternions(6, 31)
    qt = synth.perturb(ql, 5.0, 32)
    pats = orc.project_many(master, qt, pc, n).astype(np.float32)
    q, pk, it = orc.refine_many(master, pats, ql, pc, max_it=10, tol_deg=1e-3)
    err = orc.disorientation(q, qt)
    assert err.max() < 0.01
    assert np.all(it <= 8) and np.all(pk > 0.999)


def test_refine_two_iterations_and_off_centre_pc(orc, master):
    """The paper's setting: two refinement iterations bring the error from the
    library spacing to well below 0.2 deg (Fig. 8), also for a PC away from the
    screen centre (second-order terms, handled by iterating)."""
    n = 128
    pc = np.array([0.47, 0.54, 0.62])
    ql = synth.random_quaternions(6, 41)
    qt = synth.perturb(ql, 3.0, 42)
    pats = orc.project_many(master, qt, pc, n).astype(np.float32)
    q2, _, _ = orc.refine_many(master, pats, ql, pc, max_it=2, tol_deg=0.0)
    init = orc.disorientation(ql, qt)
    err = orc.disorientation(q2, qt)
    assert init.mean() > 2.0
    assert err.mean() < 0.2
