"""Eulerian grid face coordinates (cells are [face_i, face_{i+1}))."""

import numpy as np


def uniform_faces(n, lo=-1.0, hi=1.0):
    """n+1 equispaced faces on [lo, hi] (float64)."""
    return lo + (hi - lo) * np.arange(n + 1, dtype=np.float64) / n


def tanh_faces(n, beta=1.5, lo=-1.0, hi=1.0):
    """n+1 faces clustered at both ends: z(xi) = tanh(beta(2 xi - 1)) / tanh(beta), xi = i/n.

    The faces are rounded to float32 values so that single- and
    double-precision consumers locate markers against the same grid.  The end
    faces are exactly ``lo`` and ``hi``.
    """
    xi = np.arange(n + 1, dtype=np.float64) / n
    s = np.tanh(beta * (2.0 * xi - 1.0)) / np.tanh(beta)
    f = lo + (hi - lo) * 0.5 * (s + 1.0)
    f = f.astype(np.float32).astype(np.float64)
    f[0], f[-1] = lo, hi
    if np.any(np.diff(f) <= 0):
        raise ValueError("tanh faces collapse in float32; use fewer cells or a smaller beta")
    return f
