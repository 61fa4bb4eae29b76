"""Pins of the oracle's master-pattern lookup, gnomonic projector, cubic
symmetry and disorientation (SO(3) Library Generation, second Equation 6)."""
import json
import math
import os

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_lambert_roundtrip_and_equal_area(orc):
    rng = np.random.default_rng(0)
    v = rng.standard_normal((4000, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    v[:, 2] = np.abs(v[:, 2])
    XY = np.array([orc.lambert_forward(p) for p in v])
    L = math.sqrt(math.pi / 2)
    assert np.abs(XY).max() <= L + 1e-12
    back = np.array([orc.lambert_inverse(x, y) for x, y in XY])
    np.testing.assert_allclose(back, v, atol=1e-12)
    # equal area: uniform directions land uniformly on the square (chi-square, 8x8 bins)
    h, _, _ = np.histogram2d(XY[:, 0], XY[:, 1], bins=8, range=[[-L, L], [-L, L]])
    expect = len(v) / 64
    chi2 = np.sum((h - expect) ** 2 / expect)
    assert chi2 < 120  # 63 dof: p ~ 1e-5 at 120


def test_lookup_at_cell_centres_matches_grid(orc):
    """The oracle's forward map, evaluated at the directions the (independent)
    generator assigns to cell centres, lands exactly on those cells."""
    M = 64
    master = synth.master_pattern("bcc", M)
    dirs = synth.master_grid_directions(M)
    rng = np.random.default_rng(1)
    for _ in range(200):
        h, a, b = rng.integers(0, 2), rng.integers(0, M), rng.integers(0, M)
        d = dirs[h, a, b]
        if abs(d[2]) < 1e-9:
            continue
        assert orc.master_lookup(master, d) == pytest.approx(float(master[h, a, b]), rel=1e-9, abs=1e-9)


def _linear_master(M, a):
    """Master whose value is the linear function a . v of the direction."""
    d = synth.master_grid_directions(M)
    return (d @ np.asarray(a)).astype(np.float32)


def test_projection_pc_pixel_is_detector_normal(orc):
    """With master value = cos(angle to the crystal direction of the detector
    normal), the projection peaks at the pattern-centre pixel and falls off as
    L / sqrt(L^2 + r^2) with L = pcz n (gnomonic geometry)."""
    n = 64
    q = synth.random_quaternions(1, 5)[0]
    pc = np.array([0.4, 0.6, 0.7])
    R = orc.quat_to_matrix(q)
    al = math.radians(20.0)
    normal_s = np.array([0.0, -math.sin(al), math.cos(al)])    # detector z in the sample frame
    a = R @ normal_s
    img = orc.project(_linear_master(1024, a), q, pc, n)
    rows, cols = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    Ld = pc[2] * n
    r2 = (cols - pc[0] * n) ** 2 + (rows - pc[1] * n) ** 2
    err = np.abs(img - Ld / np.sqrt(Ld ** 2 + r2))
    # bilinear interpolation across the Lambert map's diagonal kink limits the
    # worst pixel; the bulk follows the closed form much more tightly
    assert err.max() < 1e-3 and np.median(err) < 2e-5


def test_projection_great_circles_are_lines(orc):
    """Gnomonic projection: the trace of a crystal plane (a great circle) is a
    straight line on the detector."""
    n = 128
    rng = np.random.default_rng(2)
    for k in range(3):
        q = synth.random_quaternions(1, 10 + k)[0]
        g = rng.standard_normal(3)
        g /= np.linalg.norm(g)
        img = orc.project(_linear_master(1024, g), q, (0.5, 0.5, 0.6), n)
        pts = []
        for i in range(n):
            row = img[i]
            s = np.where(np.sign(row[:-1]) != np.sign(row[1:]))[0]
            for j in s:
                t = row[j] / (row[j] - row[j + 1])
                pts.append((i + 0.5, j + 0.5 + t))
        for j in range(n):
            col = img[:, j]
            s = np.where(np.sign(col[:-1]) != np.sign(col[1:]))[0]
            for i in s:
                t = col[i] / (col[i] - col[i + 1])
                pts.append((i + 0.5 + t, j + 0.5))
        if len(pts) < 20:
            continue
        P = np.array(pts)
        P -= P.mean(0)
        _, s, _ = np.linalg.svd(P, full_matrices=False)
        assert s[1] / math.sqrt(len(P)) < 0.01   # rms distance to the best line < 0.01 px


def test_quat_matrix_and_cubic_group(orc):
    q = synth.random_quaternions(5, 3)
    for qq in q:
        R = orc.quat_to_matrix(qq)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0)
    Rz = orc.quat_to_matrix([math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)])
    np.testing.assert_allclose(Rz @ [1, 0, 0], [0, 1, 0], atol=1e-15)
    ops = orc.cubic_ops()
    g = json.load(open(os.path.join(GOLD, "cubic_counts.json")))
    assert len(ops) == g["n_symmetry_operators"]
    mats = [orc.quat_to_matrix(o) for o in ops]
    for A in mats:   # every operator permutes the cube axes with signs
        assert np.allclose(np.abs(A).sum(0), 1) and np.allclose(np.abs(A).sum(1), 1)
    keys = {tuple(np.round(m, 9).ravel()) for m in mats}
    assert len(keys) == 24
    for A in mats:  # closure
        for B in mats:
            assert tuple(np.round(A @ B, 9).ravel()) in keys


def test_disorientation_closed_forms(orc):
    g = json.load(open(os.path.join(GOLD, "disorientation.json")))
    for ang, expect in g["about_001"]:
        a = math.radians(ang)
        qb = np.array([math.cos(a / 2), 0, 0, math.sin(a / 2)])
        assert orc.disorientation(np.array([1.0, 0, 0, 0]), qb) == pytest.approx(expect, abs=1e-9)
    qa = synth.random_quaternions(3000, 7)
    qb = synth.random_quaternions(3000, 8)
    d = orc.disorientation(qa, qb)
    assert d.max() <= g["max_deg"] + 1e-6 and d.max() > 55.0
    ops = orc.cubic_ops()
    for i in range(24):
        assert orc.disorientation(orc.qmul(ops[i], qa[i]), qa[i]) == pytest.approx(0.0, abs=1e-6)
    # symmetric in its arguments
    assert np.allclose(orc.disorientation(qa[:50], qb[:50]), orc.disorientation(qb[:50], qa[:50]))


def test_projection_respects_crystal_symmetry(orc):
    """The master is invariant under the 24 cubic rotations, so g and S g give
    the same template up to bilinear interpolation error."""
    m = synth.master_pattern("bcc", 1024)
    q = synth.random_quaternions(1, 12)[0]
    base = orc.project(m, q, (0.5, 0.5, 0.6), 64)
    rngv = base.max() - base.min()
    for S in orc.cubic_ops()[1::5]:
        other = orc.project(m, orc.qmul(S, q), (0.5, 0.5, 0.6), 64)
        assert np.abs(other - base).max() < 0.02 * rngv


def test_generator_library_counts_near_paper(orc):
    """The S^2 x S^1 fundamental-zone generator gives the paper's library sizes
    to within a few percent (618 at 10 deg, 4958 at 5 deg)."""
    g = json.load(open(os.path.join(GOLD, "cubic_counts.json")))
    for step, count in [("10", g["counts"]["10"]), ("5", g["counts"]["5"])]:
        n = len(synth.so3_grid_cubic_fz(float(step)))
        assert abs(n - count) / count < 0.03
