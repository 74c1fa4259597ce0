"""Pins for the adaptive Lagrangian refinement oracle (Section 3, Fig. 5, Table 1)."""

import numpy as np
import pytest

import oracle
from oracle.refine import PIECES, refine, refine_levels, sub_triangles
from workloads import uniform_faces
from workloads.geometry import icosphere

RNG = np.random.default_rng(31)


def _random_triangles(n):
    V = RNG.normal(size=(3 * n, 3)) * 0.05
    V += np.repeat(RNG.uniform(-0.5, 0.5, size=(n, 3)), 3, axis=0)
    tri = np.arange(3 * n).reshape(n, 3)
    return V, tri


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_partition_area_and_first_moment(k):
    """The refined triangles tile the base triangle: their areas sum to A and the
    area-weighted mean of their centroids is the base centroid."""
    V, tri = _random_triangles(50)
    level = np.full(50, k)
    x0, a0 = oracle.marker_prep(V, tri, "f64")
    x, a, parent = refine(V, tri, level, "f64")
    assert np.array_equal(np.bincount(parent, minlength=50), np.full(50, PIECES[k]))
    asum = np.bincount(parent, weights=a, minlength=50)
    assert np.max(np.abs(asum - a0) / a0) < 1e-12
    for d in range(3):
        m = np.bincount(parent, weights=a * x[d], minlength=50) / asum
        assert np.max(np.abs(m - x0[d])) < 1e-12


def test_construction_points_of_fig5():
    """L1 is the midpoint of V1V2, L2 the centroid, L31/L32/L33 the edge midpoints."""
    V = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    tri = np.array([[0, 1, 2]])
    p1, p2, p3, _ = sub_triangles(V, tri, np.array([1]), "f64")
    assert np.allclose(p2[0], [0.5, 0.0, 0.0]) and np.allclose(p1[1], [0.5, 0.0, 0.0])
    p1, p2, p3, _ = sub_triangles(V, tri, np.array([2]), "f64")
    assert np.allclose(p3, [[1 / 3, 2 / 3, 0.0]] * 3)
    p1, p2, p3, _ = sub_triangles(V, tri, np.array([3]), "f64")
    assert np.allclose(p1[3], [0.5, 0, 0]) and np.allclose(p2[3], [0.5, 1, 0]) and np.allclose(p3[3], [0, 1, 0])
    _, a, _ = refine(V, tri, np.array([3]), "f64")
    assert np.allclose(a, 0.25)                          # four congruent quarters of area 1


def test_table1_ratios():
    """Uniform levels 1, 2, 3 multiply the marker count by 2, 3, 4 (Table 1:
    162 -> 324, 642 -> 1926, 642 -> 2568)."""
    V, tri = icosphere(3)
    n = tri.shape[0]
    for k, ratio in ((1, 2), (2, 3), (3, 4)):
        _, _, parent = refine(V, tri, np.full(n, k), "f32")
        assert parent.shape[0] == ratio * n


def test_level_rule():
    """Small elements keep level 0, large ones take more pieces; the level is
    monotone in area and capped by max_level; outside the grid it is 0."""
    grid = oracle.Grid([uniform_faces(16)] * 3, (True, True, True))
    h = 2.0 / 16
    base = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.5, np.sqrt(3) / 2, 0.0]])
    sizes = np.array([0.5, 0.8 * 1.2, 0.8 * 1.6, 0.8 * 1.9, 3.0]) * h     # edge lengths
    V = np.concatenate([base * s + 0.01 for s in sizes])
    tri = np.arange(3 * len(sizes)).reshape(-1, 3)
    lev = refine_levels(grid, V, tri, ratio=0.8, max_level=3, precision="f64")
    assert lev.tolist() == [0, 1, 2, 3, 3]
    assert refine_levels(grid, V, tri, ratio=0.8, max_level=1, precision="f64").tolist() == [0, 1, 1, 1, 1]
    V_out = V + 5.0
    assert np.all(refine_levels(grid, V_out, tri, ratio=0.8, precision="f64") == 0)
