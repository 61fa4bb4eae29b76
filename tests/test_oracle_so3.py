"""Pins of the oracle's SO(3) library generator and nearest-neighbour
disorientation study (SO(3) Library Generation and Sampling Frequency
sections, the second Eq. 6, Fig. 2): the paper's library counts and its
statements about the nearest-neighbour distribution, the fundamental zone as
the minimum-angle representatives, brute-force nearest neighbours, and
coverage of random orientations."""
import numpy as np
import pytest

import oracle as orc
import synth

IDENT = np.array([1.0, 0.0, 0.0, 0.0])


@pytest.fixture(scope="module")
def grids():
    return {sf: orc.so3_grid(sf) for sf in (10.0, 7.5)}


def test_counts_near_the_papers(grids):
    """618 orientations at 10 deg and 4,958 at 5 deg for cubic symmetry."""
    assert abs(len(grids[10.0]) - 618) <= 0.02 * 618
    n5 = len(orc.so3_grid(5.0, dedup=False))
    assert abs(n5 - 4958) <= 0.02 * 4958


def test_grid_is_the_generator_definition():
    """Without the duplicate rule the grid is the plain S^2 x S^1 construction
    (numpy restatement of the same scheme, independent code)."""
    for sf in (10.0, 7.0):
        np.testing.assert_allclose(orc.so3_grid(sf, dedup=False), synth.so3_grid_cubic_fz(sf), atol=1e-13)


def test_members_are_minimum_angle_representatives(grids):
    """The cubic zone holds the representative of each orbit with the
    smallest rotation angle: a member's own angle is its disorientation from
    the identity."""
    for g in grids.values():
        own = 2 * np.degrees(np.arccos(np.clip(np.abs(g[:, 0]), 0, 1)))
        np.testing.assert_allclose(own, orc.disorientation(g, np.tile(IDENT, (len(g), 1))), atol=1e-9)
        assert np.all(g[:, 0] >= 0)
        np.testing.assert_allclose(np.linalg.norm(g, axis=1), 1.0, atol=1e-14)


def test_duplicate_rule(grids):
    g = grids[7.5]
    raw = orc.so3_grid(7.5, dedup=False)
    ang, _ = orc.nearest_disorientation(g)
    assert ang.min() > 1e-3                      # no symmetry copies left
    a2, i2 = orc.nearest_disorientation(raw, mode=2)
    dup = (a2 >= 0) & (a2 < 1e-3)
    assert dup.sum() == len(raw) - len(g) > 0    # exactly the copies of earlier points went
    np.testing.assert_array_equal(raw[~dup], g)


def test_nearest_neighbour_matches_brute_force():
    qa = synth.random_quaternions(37, 3)
    qb = synth.random_quaternions(53, 4)
    qb[10] = qb[3]                               # equal candidates: the lower index wins
    D = np.array([[orc.disorientation(a, b) for b in qb] for a in qa])
    ang, idx = orc.nearest_disorientation(qa, qb)
    np.testing.assert_allclose(ang, D.min(1), atol=1e-12)
    np.testing.assert_array_equal(idx, D.argmin(1))
    assert not np.any(idx == 10)
    # one set: self excluded; earlier entries only
    S = np.array([[orc.disorientation(a, b) for b in qa] for a in qa])
    np.fill_diagonal(S, np.inf)
    ang1, idx1 = orc.nearest_disorientation(qa)
    np.testing.assert_allclose(ang1, S.min(1), atol=1e-12)
    np.testing.assert_array_equal(idx1, S.argmin(1))
    ang2, idx2 = orc.nearest_disorientation(qa, mode=2)
    assert ang2[0] == -1 and idx2[0] == -1
    for i in range(1, len(qa)):
        assert idx2[i] == np.argmin(S[i, :i]) and ang2[i] == pytest.approx(S[i, :i].min(), abs=1e-12)


def test_nearest_neighbour_distribution_as_the_paper_states(grids):
    """Fig. 2: the disorientation to the closest neighbour is at most the
    sampling frequency (MTEX's exceeds it by 0.182 deg at most) and fewer than
    20 % of members sit significantly closer."""
    for sf, g in grids.items():
        ang, _ = orc.nearest_disorientation(g)
        assert ang.max() <= sf + 0.182
        assert np.mean(ang < 0.9 * sf) < 0.2
        assert abs(np.median(ang) - sf) < 0.05 * sf


def test_random_orientations_are_covered(grids):
    """Every orientation has a library member within the sampling frequency
    (what the template search relies on)."""
    r = synth.random_quaternions(1500, 7)
    for sf, g in grids.items():
        ang, _ = orc.nearest_disorientation(r, g)
        assert ang.max() <= sf and ang.mean() < 0.6 * sf
