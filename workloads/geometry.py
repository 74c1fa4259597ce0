"""Triangulated synthetic bodies: icospheres, ellipsoids, deformed spheres.

Face order matters for locality only: each subdivision replaces a triangle by
its four children in place, so consecutive faces stay spatially close.
"""

import numpy as np


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
    ], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    return v, f


def icosphere(level):
    """Unit icosphere: (vertices (V,3) float64 on the unit sphere, faces (F,3) int32).

    V = 10*4**level + 2, F = 20*4**level.  Faces are counter-clockwise seen
    from outside.
    """
    v, f = _icosahedron()
    verts = [row for row in v]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            j = cache.get(key)
            if j is None:
                p = verts[a] + verts[b]
                p = p / np.linalg.norm(p)
                j = len(verts)
                verts.append(p)
                cache[key] = j
            return j

        nf = np.empty((4 * len(f), 3), dtype=np.int64)
        for n, (a, b, c) in enumerate(f):
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf[4 * n + 0] = (a, ab, ca)
            nf[4 * n + 1] = (b, bc, ab)
            nf[4 * n + 2] = (c, ca, bc)
            nf[4 * n + 3] = (ab, bc, ca)
        f = nf
    return np.asarray(verts, dtype=np.float64), f.astype(np.int32)


def random_rotation(rng):
    """Uniformly distributed rotation matrix from a uniform random unit quaternion."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def sh_basis(unit_vertices, lmax=6):
    """Real spherical-harmonic basis (nv, n_terms) for l = 1..lmax (unnormalised)."""
    from scipy.special import lpmv
    x, y, z = unit_vertices.T
    ct = np.clip(z, -1.0, 1.0)
    ph = np.arctan2(y, x)
    cols = []
    for l in range(1, lmax + 1):
        for m in range(0, l + 1):
            p = lpmv(m, l, ct)
            cols.append(p * np.cos(m * ph))
            if m > 0:
                cols.append(p * np.sin(m * ph))
    return np.stack(cols, axis=1)


def sh_radial_factor(basis, rng, amplitude=0.05):
    """Radial factor 1 + amplitude * S/max|S|, S = basis @ a with a ~ N(0,1).

    ``basis`` comes from :func:`sh_basis`; its normalisation does not matter
    because S is rescaled by its maximum over the vertices.
    """
    s = basis @ rng.normal(size=basis.shape[1])
    return 1.0 + amplitude * s / np.max(np.abs(s))


def place_bodies(rng, radii, lo, hi, gap, margin, max_tries=200000):
    """Non-overlapping centres by seeded rejection sampling.

    Each body is bounded by a sphere of radius ``radii[b]``; two bodies keep a
    clearance of ``gap`` between bounding spheres, and each sphere stays
    ``margin[d]`` away from the box faces ``lo[d]``/``hi[d]``.  A uniform bin
    grid keeps the overlap test local.
    """
    radii = np.asarray(radii, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    margin = np.asarray(margin, dtype=np.float64)
    rmax = float(radii.max())
    bin_w = 2.0 * rmax + gap
    nb = np.maximum(1, np.floor((hi - lo) / bin_w).astype(int))
    bins = {}
    centres = np.empty((len(radii), 3))
    tries = 0
    for b, r in enumerate(radii):
        while True:
            tries += 1
            if tries > max_tries:
                raise RuntimeError("body placement failed: domain too crowded")
            c = lo + margin + r + rng.random(3) * (hi - lo - 2 * (margin + r))
            key = tuple(np.minimum(((c - lo) / bin_w).astype(int), nb - 1))
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for o in bins.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                            if np.sum((centres[o] - c) ** 2) < (radii[o] + r + gap) ** 2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                centres[b] = c
                bins.setdefault(key, []).append(b)
                break
    return centres
