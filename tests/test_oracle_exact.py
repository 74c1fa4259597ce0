"""Pins for the oracle's exact-MLS shape functions (Eqs. 2-6).

Each check ties the oracle to something other than itself: a closed form
derived from Eq. 3 for separable weights, a brute-force minimisation of
Eq. 2, the invariants the method guarantees, and hand-derived special cases.
"""

import numpy as np
import pytest

import oracle
from workloads import uniform_faces, tanh_faces

RNG = np.random.default_rng(7)


def _random_markers(grid, m, rng, interior=2):
    """Markers uniformly inside cells [interior, n-1-interior) on each axis."""
    x = np.empty((3, m))
    for d in range(3):
        f = grid.faces[d]
        x[d] = rng.uniform(f[interior], f[grid.n[d] - interior], size=m)
    return x


def _grids():
    yield oracle.Grid([uniform_faces(16)] * 3, (True, True, True))
    # Non-uniform on every axis (random widths), walled.
    g = np.random.default_rng(3)
    faces = [np.concatenate([[0.0], np.cumsum(g.uniform(0.5, 1.5, size=20))]) for _ in range(3)]
    yield oracle.Grid(faces, (False, False, False))
    # The stretched-in-z grid shape of the large workload, small.
    yield oracle.Grid([uniform_faces(32), uniform_faces(32), tanh_faces(32, 1.5)], (True, True, False))


def _closed_form(grid, x, eps):
    """phi_k = prod_d (w_d/mu0_d) * (1 - sum_d m_d (xi_kd - m_d)/v_d).

    With a separable weight and a tensor-product 3x3x3 stencil the moment
    matrix of Eq. 3 factorises per axis into moments mu0, mu1, mu2 of the
    1-D weights over the 3 nodes; m = mu1/mu0 and v = mu2/mu0 - m^2.  Solving
    Eq. 6 with that factorised A gives this formula (derived independently of
    the oracle's assembly and solve).
    """
    M = x.shape[1]
    phi = np.ones((M, 27))
    corr = np.ones((M, 27))
    offs = np.array([(ax, ay, az) for az in (-1, 0, 1) for ay in (-1, 0, 1) for ax in (-1, 0, 1)])
    for d in range(3):
        f, n = grid.faces[d], grid.n[d]
        c = 0.5 * (f[:-1] + f[1:])
        w = np.diff(f)
        i = np.searchsorted(f, x[d], side="right") - 1
        xi = np.empty((M, 3))
        for a in (-1, 0, 1):
            j = i + a
            xi[:, a + 1] = (c[j] - x[d]) / w[i]
        wd = np.exp(-xi ** 2 / eps ** 2)
        mu0, mu1, mu2 = wd.sum(1), (wd * xi).sum(1), (wd * xi ** 2).sum(1)
        m, v = mu1 / mu0, mu2 / mu0 - (mu1 / mu0) ** 2
        sel = offs[:, d] + 1
        phi *= wd[:, sel] / mu0[:, None]
        corr -= m[:, None] * (xi[:, sel] - m[:, None]) / v[:, None]
    return phi * corr


@pytest.mark.parametrize("eps", [0.7, 1.0, 1.6])
def test_closed_form_separable(eps):
    for grid in _grids():
        x = _random_markers(grid, 400, RNG)
        tr = oracle.shape_exact(grid, x, eps)
        assert tr.sup.ok.all()
        ref = _closed_form(grid, x, eps)
        assert np.max(np.abs(tr.phi - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_brute_force_least_squares():
    """Minimise J of Eq. 2 directly for q = unit vectors; Q(x_l) is phi_k."""
    for grid in _grids():
        x = _random_markers(grid, 25, RNG)
        tr = oracle.shape_exact(grid, x, 1.0)
        for m in range(x.shape[1]):
            pos = tr.sup.pos[:, m, :]                      # (3, 27)
            w = np.exp(-sum(((pos[d] - x[d, m]) / tr.sup.hwidth[d, m]) ** 2 for d in range(3)))
            P = np.stack([np.ones(27), pos[0], pos[1], pos[2]], axis=1)
            sw = np.sqrt(w)[:, None]
            for k in range(27):
                q = np.zeros(27)
                q[k] = 1.0
                a, *_ = np.linalg.lstsq(sw * P, sw[:, 0] * q, rcond=None)
                Q = np.array([1.0, x[0, m], x[1, m], x[2, m]]) @ a
                assert abs(Q - tr.phi[m, k]) < 1e-9


def test_partition_of_unity_and_linear_reproduction():
    for grid in _grids():
        x = _random_markers(grid, 500, RNG)
        tr = oracle.shape_exact(grid, x, 1.0)
        assert np.max(np.abs(tr.phi.sum(1) - 1.0)) < 1e-13
        for d in range(3):
            rep = np.sum(tr.phi * tr.sup.pos[d], axis=1)
            scale = np.max(np.abs(grid.faces[d]))
            assert np.max(np.abs(rep - x[d])) < 1e-13 * scale


def test_absolute_basis_matches_centred_basis():
    grid = oracle.Grid([uniform_faces(8, 0.0, 1.0)] * 3, (True, True, True))
    x = _random_markers(grid, 200, RNG, interior=0)
    a = oracle.shape_exact(grid, x, 1.0).phi
    b = oracle.shape_exact_absolute_basis(grid, x, 1.0).phi
    assert np.max(np.abs(a - b)) < 1e-10


def test_translation_invariance_whole_cells():
    """Markers at the same relative position in their cells share phi (Section 2)."""
    grid = oracle.Grid([uniform_faces(16)] * 3, (True, True, True))
    h = 2.0 / 16
    x = _random_markers(grid, 100, RNG, interior=3)
    a = oracle.shape_exact(grid, x, 1.0).phi
    for shift in [(1, 0, 0), (0, -2, 0), (3, 1, -1)]:
        xs = x + h * np.array(shift, dtype=float)[:, None]
        b = oracle.shape_exact(grid, xs, 1.0).phi
        assert np.max(np.abs(a - b)) < 1e-12


def test_marker_at_cell_centre_closed_form():
    """At a cell centre of a uniform grid the moment matrix is diagonal: phi_k = W_k / sum W."""
    grid = oracle.Grid([uniform_faces(10)] * 3, (True, True, True))
    x = np.array([[grid.centres[0][4]], [grid.centres[1][5]], [grid.centres[2][6]]])
    for eps in (0.8, 1.0):
        phi = oracle.shape_exact(grid, x, eps).phi[0]
        e = np.exp(-1.0 / eps ** 2)
        # Node weight = e^(number of non-zero offsets); sum = (1 + 2e)^3.
        nz = np.array([abs(ax) + abs(ay) + abs(az)
                       for az in (-1, 0, 1) for ay in (-1, 0, 1) for ax in (-1, 0, 1)])
        ref = e ** nz / (1.0 + 2.0 * e) ** 3
        assert np.max(np.abs(phi - ref)) < 1e-15
    # eps = 1: centre weight 1/(1 + 2/e)^3, a hand-computed number.
    phi = oracle.shape_exact(grid, x, 1.0).phi[0]
    assert abs(phi[13] - 0.19121933828981982) < 1e-14


def test_periodic_wrap_and_walls():
    n = 12
    grid = oracle.Grid([uniform_faces(n)] * 3, (True, True, True))
    h = 2.0 / n
    t = np.array([0.31, -0.22, 0.05])
    x_edge = np.array([-1.0 + (0.5 + t[0]) * h, -1.0 + (n - 0.5 + t[1]) * h, (0.5 + t[2]) * h])[:, None]
    x_mid = np.array([-1.0 + (5.5 + t[0]) * h, -1.0 + (5.5 + t[1]) * h, (0.5 + t[2]) * h])[:, None]
    a = oracle.shape_exact(grid, x_edge, 1.0)
    b = oracle.shape_exact(grid, x_mid, 1.0)
    assert np.max(np.abs(a.phi - b.phi)) < 1e-12
    assert set(a.sup.idx[0, 0]) == {n - 1, 0, 1}
    assert set(a.sup.idx[1, 0]) == {n - 2, n - 1, 0}
    walled = oracle.Grid([uniform_faces(n)] * 3, (True, True, False))
    xw = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [-1.0 + 0.5 * h, -1.0 + 1.5 * h, 1.0 - 0.5 * h]])
    home, ok = oracle.locate(walled, xw)
    assert list(ok) == [False, True, False]
    # Outside the box or non-finite: not usable.
    bad = np.array([[1.0, np.nan, 0.0], [0.0, 0.0, -1.5], [0.0, 0.0, 0.0]])
    _, ok = oracle.locate(grid, bad)
    assert not ok.any()


def test_home_cell_half_open():
    grid = oracle.Grid([uniform_faces(8)] * 3, (True, True, True))
    f = grid.faces[0]
    x = np.array([[f[3], np.nextafter(f[3], -np.inf), f[0]], [0.0] * 3, [0.0] * 3])
    home, ok = oracle.locate(grid, x)
    assert list(home[0]) == [3, 2, 0] and ok.all()


def test_moment_matrix_pins():
    """A of Eq. 3: diagonal at a uniform cell centre with closed-form entries
    (sum W = (1 + 2e)^3, sum W xi_d^2 = 2e (1 + 2e)^2 at eps = 1, e = exp(-1)),
    so cond_1 = (1 + 2e) / (2e); A^-1 e_0 reproduces shape_exact's phi; and the
    conditioning grows without bound as a cell's neighbours get wider."""
    grid = oracle.Grid([uniform_faces(10)] * 3, (True, True, True))
    x = np.array([[grid.centres[0][4]], [grid.centres[1][5]], [grid.centres[2][6]]])
    A, cond = oracle.moment_matrix(grid, x, 1.0)
    e = np.exp(-1.0)
    ref = np.diag([(1 + 2 * e) ** 3] + [2 * e * (1 + 2 * e) ** 2] * 3)
    assert np.max(np.abs(A[0] - ref)) < 1e-14
    assert abs(cond[0] - (1 + 2 * e) / (2 * e)) < 1e-13
    g2 = oracle.Grid([uniform_faces(12), uniform_faces(12), tanh_faces(12, 1.5)], (True, True, False))
    rng = np.random.default_rng(4)
    xs = np.stack([rng.uniform(-0.8, 0.8, 30) for _ in range(3)])
    A, cond = oracle.moment_matrix(g2, xs, 1.0)
    y = np.linalg.solve(A, np.tile([1.0, 0, 0, 0], (30, 1))[:, :, None])[:, :, 0]
    sup = oracle.support(g2, xs)
    W = oracle.gaussian_weight(xs, sup, 1.0)
    xi = np.stack([(sup.pos[d] - xs[d][:, None]) / sup.hwidth[d][:, None] for d in range(3)])
    P = oracle.basis_values(xi)
    phi = W * np.einsum("mki,mi->mk", P, y)
    assert np.max(np.abs(phi - oracle.shape_exact(g2, xs, 1.0).phi)) < 1e-13
    assert np.all(cond >= 1.0)
    med = []
    for r in (1.0, 3.0, 5.0, 8.0):
        w = np.array([r, r, r, 1.0, r, r, r])
        fz = np.concatenate([[0.0], np.cumsum(w)])
        fz = fz / fz[-1] * 2 - 1
        g3 = oracle.Grid([uniform_faces(8), uniform_faces(8), fz], (True, True, False))
        xz = np.stack([rng.uniform(-0.5, 0.5, 50), rng.uniform(-0.5, 0.5, 50), rng.uniform(fz[3], fz[4], 50)])
        med.append(np.median(oracle.moment_matrix(g3, xz, 1.0)[1]))
    assert all(a < b for a, b in zip(med, med[1:])) and med[-1] > 1e6
