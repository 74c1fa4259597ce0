"""Pins for marker preparation: triangle centroids and areas (Section 3, Eq. 7)."""

import numpy as np

import oracle
from workloads import icosphere


def test_known_triangles():
    V = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [2, 0, 0], [3, 0, 0], [2.5, np.sqrt(3) / 2, 0],
                  [0, 0, 1], [0, 2, 1], [0, 0, 4]])
    T = np.array([[0, 1, 2], [3, 4, 5], [6, 7, 8]], dtype=np.int32)
    c, a = oracle.marker_prep(V, T)
    assert np.allclose(c[:, 0], [1 / 3, 1 / 3, 0], atol=1e-15)
    assert np.allclose(c[:, 1], [2.5, np.sqrt(3) / 6, 0], atol=1e-15)
    assert np.allclose(c[:, 2], [0, 2 / 3, 2], atol=1e-15)
    assert np.allclose(a, [0.5, np.sqrt(3) / 4, 3.0], atol=1e-15)


def test_icosphere_area_converges_to_sphere():
    R = 0.7
    prev = 0.0
    for level in range(5):
        v, f = icosphere(level)
        _, a = oracle.marker_prep(R * v, f)
        total = a.sum()
        assert prev < total < 4 * np.pi * R ** 2        # inscribed flat faces, monotone
        prev = total
    assert abs(prev / (4 * np.pi * R ** 2) - 1) < 5e-3


def test_icosahedron_area_closed_form():
    # Unit circumradius icosahedron: edge a = 4/sqrt(10 + 2 sqrt 5); area 5 sqrt(3) a^2.
    v, f = icosphere(0)
    _, a = oracle.marker_prep(v, f)
    edge = 4.0 / np.sqrt(10 + 2 * np.sqrt(5))
    assert abs(a.sum() - 5 * np.sqrt(3) * edge ** 2) < 1e-13
    # Closed centred surface: area-weighted centroids sum to zero.
    c, a = oracle.marker_prep(v, f)
    assert np.max(np.abs((c * a).sum(1))) < 1e-14


def test_single_precision_prep_error_bound():
    """The fixed-order float32 evaluation stays within a few ulps of the float64 definition."""
    g = np.random.default_rng(3)
    v, f = icosphere(3)
    V = 0.02 * v + g.uniform(-0.9, 0.9, size=3)
    V32 = V.astype(np.float32).astype(np.float64)
    c64, a64 = oracle.marker_prep(V32, f, "f64")
    c32, a32 = oracle.marker_prep(V32, f, "f32")
    ulp = np.spacing(np.abs(c64).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(c32 - c64) <= 2.0 * ulp)
    # Area: cancellation in the edge vectors is exact (Sterbenz), so the
    # relative error is a few float32 roundings.
    assert np.max(np.abs(a32 - a64) / a64) < 1e-6
