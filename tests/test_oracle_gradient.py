"""Pins for the exact-MLS shape-function gradients (derivative of Eq. 6).

Checked against central finite differences of the shape functions themselves
(an independent route through the dense solve of Eq. 6), against the
identities the linear basis fixes (sum_k d_d phi_k = 0 and
sum_k d_d phi_k x_k,e = delta_de, the derivatives of Eq. 6's exact linear
reproduction), and against exact gradients of linear velocity fields.
"""

import numpy as np
import pytest

import oracle
from workloads import tanh_faces, uniform_faces

RNG = np.random.default_rng(41)


def _grids():
    yield oracle.Grid([uniform_faces(12)] * 3, (True, True, True))
    yield oracle.Grid([uniform_faces(12), uniform_faces(14), tanh_faces(16, 1.5)], (True, True, False))


def _markers(grid, m):
    x = np.empty((3, m))
    for d in range(3):
        f = grid.faces[d]
        x[d] = RNG.uniform(f[2], f[grid.n[d] - 2], size=m)
    return x


def test_matches_central_differences():
    for grid in _grids():
        x = _markers(grid, 60)
        home, _ = oracle.locate(grid, x)
        dphi = oracle.shape_exact_gradient(grid, x, 1.0)
        for d in range(3):
            delta = 1e-6 * grid.widths[d][home[d]]
            xp, xm = x.copy(), x.copy()
            xp[d] += delta
            xm[d] -= delta
            fd = (oracle.shape_exact(grid, xp, 1.0, home=home).phi
                  - oracle.shape_exact(grid, xm, 1.0, home=home).phi) / (2 * delta[:, None])
            scale = np.max(np.abs(dphi[:, d]))
            assert np.max(np.abs(fd - dphi[:, d])) < 1e-7 * scale


def test_linear_reproduction_identities():
    for grid in _grids():
        x = _markers(grid, 100)
        dphi = oracle.shape_exact_gradient(grid, x, 1.0)
        sup = oracle.support(grid, x)
        for d in range(3):
            s0 = dphi[:, d].sum(axis=1)
            scale = np.max(np.abs(dphi[:, d]))
            assert np.max(np.abs(s0)) < 1e-11 * scale
            for e in range(3):
                s1 = np.sum(dphi[:, d] * sup.pos[e], axis=1)
                assert np.max(np.abs(s1 - (1.0 if d == e else 0.0))) < 1e-11 * scale


def test_linear_field_gradient_exact():
    for grid in _grids():
        x = _markers(grid, 80)
        tr = oracle.shape_exact(grid, x, 1.0)
        dphi = oracle.shape_exact_gradient(grid, x, 1.0)
        a = RNG.normal(size=3)
        Bm = RNG.normal(size=(3, 3))
        zc, yc, xc = grid.centres[2], grid.centres[1], grid.centres[0]
        Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
        u = np.stack([a[c] + Bm[c, 0] * X + Bm[c, 1] * Y + Bm[c, 2] * Z for c in range(3)])
        G = oracle.interpolate_gradient(dphi, tr.sup, u)
        # periodic axes wrap the field, so keep markers whose stencil does not cross a seam
        inner = np.ones(x.shape[1], dtype=bool)
        for d in range(3):
            inner &= (tr.sup.home[d] >= 1) & (tr.sup.home[d] <= grid.n[d] - 2)
        assert inner.sum() > 50
        assert np.max(np.abs(G[:, :, inner] - Bm[:, :, None])) < 1e-10 * np.max(np.abs(Bm))


def test_unusable_markers_are_zero():
    grid = oracle.Grid([uniform_faces(8)] * 3, (True, True, False))
    x = np.array([[0.1], [0.2], [-0.99]])
    assert np.all(oracle.shape_exact_gradient(grid, x, 1.0) == 0)
