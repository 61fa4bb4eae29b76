"""Pins of the oracle's master interpolation: the bicubic (Keys, a = -1/2)
reading of the paper's reprojection interpolates the cell centres, reproduces
quadratics exactly away from the edges, and agrees with the bilinear lookup
on linear data; the projector with bicubic lookup stays within the
interpolation error of the bilinear one on a smooth master."""
import numpy as np

import synth


def test_interpolates_cell_centres(orc):
    rng = np.random.default_rng(0)
    g = rng.normal(size=(12, 12)).astype(np.float32)
    for (i, j) in [(0, 0), (5, 7), (11, 3), (11, 11)]:
        assert orc.grid_interp(g, j, i, 1) == np.float64(g[i, j])
        assert orc.grid_interp(g, j, i, 0) == np.float64(g[i, j])


def test_reproduces_quadratics_in_the_interior(orc):
    M = 16
    y, x = np.mgrid[0:M, 0:M].astype(np.float64)
    g = (0.3 + 0.2 * x - 0.1 * y + 0.05 * x * x - 0.02 * x * y + 0.03 * y * y).astype(np.float32)
    rng = np.random.default_rng(1)
    for fx, fy in rng.uniform(2.0, M - 3.0, size=(20, 2)):
        exact = 0.3 + 0.2 * fx - 0.1 * fy + 0.05 * fx * fx - 0.02 * fx * fy + 0.03 * fy * fy
        # the grid holds float32 values: compare to the interpolant of those values
        assert abs(orc.grid_interp(g, fx, fy, 1) - exact) < 1e-5, (fx, fy)


def test_agrees_with_bilinear_on_linear_data(orc):
    M = 10
    y, x = np.mgrid[0:M, 0:M].astype(np.float64)
    g = (1.0 + 0.5 * x + 0.25 * y).astype(np.float32)
    for fx, fy in [(2.3, 4.7), (5.5, 5.5), (3.01, 6.99)]:
        assert abs(orc.grid_interp(g, fx, fy, 1) - orc.grid_interp(g, fx, fy, 0)) < 1e-6


def test_bicubic_projection_close_to_bilinear(orc):
    master = synth.master_pattern("bcc", 512)
    q = synth.random_quaternions(2, 3)
    a = orc.project_many(master, q, (0.5, 0.5, 0.6), 64, interp=0)
    b = orc.project_many(master, q, (0.5, 0.5, 0.6), 64, interp=1)
    assert np.abs(a - b).max() < 0.05 * (a.max() - a.min())
    assert np.abs(a - b).max() > 0                      # the two lookups do differ
