"""The pins have teeth: plausible mistakes planted in the oracle (on the CPU) fail them.

Each case monkeypatches one oracle function with a wrong variant and checks
that the corresponding pin's comparison no longer holds.
"""

import numpy as np

import oracle
import oracle.mls as om
from workloads import uniform_faces, tanh_faces

from test_oracle_exact import _closed_form, _random_markers


def _stretched():
    return oracle.Grid([uniform_faces(32), uniform_faces(32), tanh_faces(32, 1.5)], (True, True, False))


def test_dropped_support_node_is_caught(monkeypatch):
    grid = _stretched()
    x = _random_markers(grid, 50, np.random.default_rng(1))
    real = om.gaussian_weight

    def dropped(xx, sup, eps):
        w = real(xx, sup, eps)
        w[:, 26] = 0.0                                     # one node missing from Eqs. 3-4
        return w

    monkeypatch.setattr(om, "gaussian_weight", dropped)
    phi = oracle.shape_exact(grid, x, 1.0).phi
    # Partition of unity still holds over the remaining nodes ...
    assert np.max(np.abs(phi.sum(1) - 1)) < 1e-12
    # ... but the closed form over all 27 nodes does not.
    assert np.max(np.abs(phi - _closed_form(grid, x, 1.0))) > 1e-4


def test_wrong_distance_scale_is_caught(monkeypatch):
    grid = _stretched()
    x = _random_markers(grid, 50, np.random.default_rng(2))

    def node_scaled(xx, sup, eps):
        r2 = sum(((sup.pos[d] - xx[d][:, None]) / sup.width[d]) ** 2 for d in range(3))
        return np.exp(-r2 / eps ** 2)                      # node width instead of home width

    monkeypatch.setattr(om, "gaussian_weight", node_scaled)
    phi = oracle.shape_exact(grid, x, 1.0).phi
    assert np.max(np.abs(phi - _closed_form(grid, x, 1.0))) > 1e-4


def test_garbled_shepard_numerator_is_caught(monkeypatch):
    """Eq. 10 as printed (numerator 1/d_j^2 with a fixed j) breaks partition of unity."""
    grid = oracle.Grid([uniform_faces(12)] * 3, (True, True, True))
    g = np.random.default_rng(3)
    x = _random_markers(grid, 40, g)
    # Replace alpha_i by (1/d_0^2)/sum_j(1/d_j^2) for every i.
    src = om.shape_fast

    def garbled(grid_, x_, eps=1.0, n_sub=9, home=None, subcell=None, tables=None):
        tr = src(grid_, x_, eps, n_sub, home, subcell, tables)
        # Recompute with the printed numerator for a direct comparison.
        out = tr.phi.copy()
        sup = tr.sup
        nm1 = n_sub - 1
        for m in range(x_.shape[1]):
            t = (x_[:, m] - np.array([grid_.faces[d][sup.home[d, m]] for d in range(3)])) / sup.hwidth[:, m] - 0.5
            u = (t + 0.5) * nm1
            s = np.minimum(np.floor(u), nm1 - 1).astype(int)
            lam = u - s
            corners = [(cx, cy, cz) for cz in (0, 1) for cy in (0, 1) for cx in (0, 1)]
            d2 = np.array([sum(((lam[d] - c[d]) / nm1) ** 2 for d in range(3)) for c in corners])
            alpha = np.full(8, (1 / d2[0]) / np.sum(1 / d2))
            key = om._table_key(grid_, sup.home[:, m])
            T = om.fast_table(grid_, key, n_sub, eps)
            nodes = [((s[2] + c[2]) * n_sub + (s[1] + c[1])) * n_sub + (s[0] + c[0]) for c in corners]
            out[m] = alpha @ T[nodes]
        return om.Transfer(out, sup)

    monkeypatch.setattr(oracle, "shape_fast", garbled)
    phi = oracle.shape_fast(grid, x, 1.0, 5).phi
    assert np.max(np.abs(phi.sum(1) - 1.0)) > 1e-3


def test_mirrored_spread_index_is_caught():
    """Spreading with the node offsets mirrored breaks adjointness with interpolation."""
    grid = oracle.Grid([uniform_faces(12)] * 3, (True, True, True))
    g = np.random.default_rng(4)
    x = _random_markers(grid, 100, g, interior=1)
    tr = oracle.shape_exact(grid, x, 1.0)
    c = np.full(100, 0.3)
    u = g.normal(size=(3, 12, 12, 12))
    F = g.normal(size=(3, 100))
    U = oracle.interpolate(tr, u)
    bad = om.Transfer(tr.phi[:, ::-1].copy(), tr.sup)      # phi_k paired with node 26-k
    f_bad = oracle.spread(bad, c, F, grid.n).to_dense(grid.n)
    f_ok = oracle.spread(tr, c, F, grid.n).to_dense(grid.n)
    assert abs(np.sum(U * c * F) - np.sum(u * f_ok)) < 1e-10
    assert abs(np.sum(U * c * F) - np.sum(u * f_bad)) > 1e-3


def test_missing_area_in_scale_is_caught():
    grid = oracle.Grid([uniform_faces(10)] * 3, (True, True, True))
    x = _random_markers(grid, 20, np.random.default_rng(5), interior=0)
    tr = oracle.shape_exact(grid, x, 1.0)
    area = np.full(20, 0.01)
    h = 0.2
    w = tr.sup.width
    h_l = np.sum(tr.phi * (w[0] + w[1] + w[2]), axis=1) / 3.0
    wrong = h_l / np.sum(tr.phi * w[0] * w[1] * w[2], axis=1)   # A_l dropped from dV_l
    assert np.max(np.abs(oracle.forcing_scale(tr, area) - area / h ** 2)) < 1e-12
    assert np.max(np.abs(wrong - area / h ** 2)) > 1.0


def test_quadratic_basis_with_a_wrong_cross_term_is_caught(monkeypatch):
    """A cross term written as xy where zx belongs still fits data but fails reproduction of zx."""
    grid = _stretched()
    x = _random_markers(grid, 30, np.random.default_rng(6))
    real = om.basis_values

    def garbled(xi, m=4):
        p = real(xi, m)
        if m == 10:
            p = p.copy()
            p[..., 9] = xi[0] * xi[1] * xi[1]              # a cubic where z*x belongs
        return p

    monkeypatch.setattr(om, "basis_values", garbled)
    tr = oracle.shape_exact(grid, x, 1.0, basis=10)
    rel = [(tr.sup.pos[d] - x[d][:, None]) / tr.sup.hwidth[d][:, None] for d in range(3)]
    zx = np.sum(tr.phi * rel[2] * rel[0], axis=1)
    assert np.max(np.abs(zx)) > 1e-3
