"""Adaptive Lagrangian refinement of the forcing markers (Section 3), plain CPU.

Test infrastructure only: the GPU library never imports this module.

A base triangle (V1, V2, V3) is split for the forcing step only (Fig. 5):
  level 0: the triangle itself;
  level 1: two triangles through L1 = (V1 + V2)/2: (V1, L1, V3), (L1, V2, V3);
  level 2: three triangles through the centroid L2: (V1, V2, L2), (V2, V3, L2),
           (V3, V1, L2);
  level 3: four triangles through the edge midpoints L31 = (V1 + V2)/2,
           L32 = (V2 + V3)/2, L33 = (V3 + V1)/2: (V1, L31, L33),
           (L31, V2, L32), (L33, L32, V3), (L31, L32, L33).
Each refined triangle contributes one marker at its centroid with its area
(the same marker definition as for base triangles), so the refined/base
ratios are 2, 3 and 4 (the uniform rows of Table 1).

Reading of the level choice (the paper says only that the refined mesh
follows the local Eulerian resolution, with element sizes of 0.7-0.9 grid
cells): the element length l is that of the equilateral triangle of the same
area, l^2 = 4 A / sqrt(3); the local spacing h is the smallest width of the
home cell of the base centroid; the level is the smallest k <= max_level
whose pieces (1, 2, 3 or 4 of them) satisfy l^2 / pieces <= (ratio h)^2,
else max_level.  A centroid outside the grid keeps level 0.  The comparison
is made in double precision on the single-precision area, as the library
does, so that both take the same integer decision.
"""

import numpy as np

from .mls import marker_prep

PIECES = (1, 2, 3, 4)
LENGTH2_PER_AREA = 4.0 / np.sqrt(3.0)


def _home_cells(grid, x):
    """Cell containing each point (no support requirement); -1 outside."""
    home = np.empty((3, x.shape[1]), dtype=np.int64)
    inside = np.all(np.isfinite(x), axis=0)
    for d in range(3):
        xd = np.where(np.isfinite(x[d]), x[d], grid.faces[d][0] - 1.0)
        i = np.searchsorted(grid.faces[d], xd, side="right") - 1
        inside &= (i >= 0) & (i < grid.n[d])
        home[d] = np.clip(i, 0, grid.n[d] - 1)
    return home, inside


def refine_levels(grid, vertices, tri, ratio=0.8, max_level=3, precision="f32"):
    """Refinement level of every base triangle (the reading above)."""
    x, area = marker_prep(vertices, tri, precision)
    home, inside = _home_cells(grid, np.asarray(x, dtype=np.float64))
    h = np.min(np.stack([grid.widths[d][home[d]] for d in range(3)]), axis=0)
    s = np.asarray(area, dtype=np.float64) * LENGTH2_PER_AREA
    rh = ratio * h
    t = rh * rh
    level = np.full(s.shape, max_level, dtype=np.int64)
    for k in range(max_level, -1, -1):
        level = np.where(s <= PIECES[k] * t, k, level)
    level[~inside | ~np.isfinite(s)] = 0
    return level


def sub_triangles(vertices, tri, level, precision="f32"):
    """Vertex coordinates of the refined triangles, in the order of the module
    docstring, and the index of their base triangle.

    Returns (P1, P2, P3) each (K, 3) and parent (K,).
    """
    dt = np.float64 if precision == "f64" else np.float32
    V = np.asarray(vertices).astype(dt)
    t = np.asarray(tri, dtype=np.int64)
    half = dt(0.5)
    out1, out2, out3, parent = [], [], [], []
    for b in range(t.shape[0]):
        v1, v2, v3 = V[t[b, 0]], V[t[b, 1]], V[t[b, 2]]
        k = int(level[b])
        if k == 0:
            subs = [(v1, v2, v3)]
        elif k == 1:
            l1 = (v1 + v2) * half
            subs = [(v1, l1, v3), (l1, v2, v3)]
        elif k == 2:
            l2 = ((v1 + v2) + v3) / dt(3)
            subs = [(v1, v2, l2), (v2, v3, l2), (v3, v1, l2)]
        else:
            l31, l32, l33 = (v1 + v2) * half, (v2 + v3) * half, (v3 + v1) * half
            subs = [(v1, l31, l33), (l31, v2, l32), (l33, l32, v3), (l31, l32, l33)]
        for p1, p2, p3 in subs:
            out1.append(p1)
            out2.append(p2)
            out3.append(p3)
            parent.append(b)
    return np.array(out1, dtype=dt), np.array(out2, dtype=dt), np.array(out3, dtype=dt), np.array(parent)


def refine(vertices, tri, level, precision="f32"):
    """Refined markers: (x (3, K), area (K,), parent (K,)), centroid and area of
    every refined triangle as for base markers."""
    p1, p2, p3, parent = sub_triangles(vertices, tri, level, precision)
    K = p1.shape[0]
    V = np.concatenate([p1, p2, p3])
    t = np.stack([np.arange(K), K + np.arange(K), 2 * K + np.arange(K)], axis=1)
    x, area = marker_prep(V, t, precision)
    return x, area, parent
