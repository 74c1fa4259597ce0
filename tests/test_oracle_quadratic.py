"""Pins for the oracle's exact-MLS shape functions with the quadratic basis.

Section 2 builds the basis p from Pascal's pyramid and leaves its size m free
(the paper uses m = 4; the fast-MLS construction does not depend on m).  For
m = 10, p = [1, x, y, z, x^2, y^2, z^2, xy, yz, zx].  The checks tie the
oracle to the definition and to mathematics:

  * a direct weighted least-squares minimisation of J (Eq. 2) in the paper's
    absolute coordinates, by a library least-squares routine (not the normal
    equations of Eq. 3 the oracle solves);
  * exact reproduction of every polynomial of degree <= 2 (the defining
    property of an MLS approximation with a complete quadratic basis);
  * a closed form at a cell centre of a uniform grid, derived by hand from
    the symmetry of the stencil;
  * the linear basis visibly failing quadratic reproduction (so the pins
    distinguish the two bases).
"""

import numpy as np
import pytest

import oracle
from workloads import tanh_faces, uniform_faces

RNG = np.random.default_rng(23)


def _grids():
    yield oracle.Grid([uniform_faces(12)] * 3, (True, True, True))
    g = np.random.default_rng(5)
    faces = [np.concatenate([[0.0], np.cumsum(g.uniform(0.5, 1.5, size=14))]) for _ in range(3)]
    yield oracle.Grid(faces, (False, False, False))
    yield oracle.Grid([uniform_faces(16), uniform_faces(16), tanh_faces(24, 1.5)], (True, True, False))


def _markers(grid, m, rng):
    x = np.empty((3, m))
    for d in range(3):
        f = grid.faces[d]
        x[d] = rng.uniform(f[2], f[grid.n[d] - 2], size=m)
    return x


def _monomials(v):
    """The ten monomials of degree <= 2 of the points v (3, N) -> (N, 10), by name."""
    x, y, z = v
    return np.stack([np.ones_like(x), x, y, z, x * x, y * y, z * z, x * y, y * z, z * x], axis=1)


def test_brute_force_weighted_least_squares():
    """phi_k(x_l) is the value at x_l of the J-minimising quadratic fitted to data e_k."""
    for grid in _grids():
        x = _markers(grid, 15, RNG)
        tr = oracle.shape_exact(grid, x, 1.0, basis=10)
        assert tr.sup.ok.all()
        origin = np.array([grid.faces[d][0] for d in range(3)])
        for m in range(x.shape[1]):
            pos = tr.sup.pos[:, m, :]                                  # (3, 27)
            w = np.exp(-sum(((pos[d] - x[d, m]) / tr.sup.hwidth[d, m]) ** 2 for d in range(3)))
            P = _monomials(pos - origin[:, None])                      # absolute coordinates
            sw = np.sqrt(w)
            a, *_ = np.linalg.lstsq(sw[:, None] * P, np.diag(sw), rcond=None)   # (10, 27), one fit per e_k
            q = _monomials((x[:, m] - origin)[:, None])[0]
            ref = q @ a
            assert np.max(np.abs(ref - tr.phi[m])) < 1e-8, np.max(np.abs(ref - tr.phi[m]))


def test_reproduces_every_quadratic():
    for grid in _grids():
        x = _markers(grid, 300, RNG)
        tr = oracle.shape_exact(grid, x, 1.0, basis=10)
        for m in range(x.shape[1]):
            h = tr.sup.hwidth[:, m]
            rel = (tr.sup.pos[:, m, :] - x[:, m][:, None]) / h[:, None]   # node offsets in home widths
            rep = tr.phi[m] @ _monomials(rel)                              # sum_k phi_k q(x_k - x_l)
            ref = np.zeros(10)
            ref[0] = 1.0                                                   # q(0)
            assert np.max(np.abs(rep - ref)) < 1e-12, rep - ref


def test_linear_basis_misses_quadratics():
    grid = next(_grids())
    x = _markers(grid, 50, RNG)
    lin = oracle.shape_exact(grid, x, 1.0, basis=4)
    h = lin.sup.hwidth[0]
    rel = (lin.sup.pos[0] - x[0][:, None]) / h[:, None]
    # sum_k phi_k (x_k - x_l)^2 is the second moment of the linear fit: well away from 0.
    assert np.min(np.sum(lin.phi * rel ** 2, axis=1)) > 0.1


@pytest.mark.parametrize("eps", [0.8, 1.0, 1.4])
def test_cell_centre_closed_form(eps):
    """At a cell centre of a uniform grid only the even terms 1, x^2, y^2, z^2 couple.

    With e = exp(-1/eps^2) the per-axis moments of the weights over the nodes
    -1, 0, 1 are m0 = 1 + 2e, m2 = m4 = 2e (odd ones vanish).  The reduced
    system A [alpha, beta, beta, beta] = e_0 (beta shared by symmetry) reads
      m0^3 alpha + 3 m2 m0^2 beta = 1,
      m2 m0^2 alpha + (m4 m0^2 + 2 m2^2 m0) beta = 0,
    and phi_k = W_k (alpha + beta n_k) with n_k the number of non-zero
    offsets of node k and W_k = e^{n_k}.
    """
    grid = oracle.Grid([uniform_faces(10)] * 3, (True, True, True))
    x = np.array([[grid.centres[0][4]], [grid.centres[1][5]], [grid.centres[2][6]]])
    phi = oracle.shape_exact(grid, x, eps, basis=10).phi[0]
    e = np.exp(-1.0 / eps ** 2)
    m0, m2, m4 = 1.0 + 2.0 * e, 2.0 * e, 2.0 * e
    S = np.array([[m0 ** 3, 3.0 * m2 * m0 ** 2],
                  [m2 * m0 ** 2, m4 * m0 ** 2 + 2.0 * m2 ** 2 * m0]])
    alpha, beta = np.linalg.solve(S, [1.0, 0.0])
    nz = np.array([abs(ax) + abs(ay) + abs(az)
                   for az in (-1, 0, 1) for ay in (-1, 0, 1) for ax in (-1, 0, 1)])
    ref = e ** nz * (alpha + beta * nz)
    assert np.max(np.abs(phi - ref)) < 1e-14


def test_same_as_linear_where_the_quadratic_terms_vanish():
    """On data that is itself linear, both bases interpolate it exactly."""
    grid = next(_grids())
    x = _markers(grid, 100, RNG)
    q = oracle.shape_exact(grid, x, 1.0, basis=10)
    g = np.array([0.3, -1.2, 0.7])
    data = np.einsum("d,dmk->mk", g, q.sup.pos) + 2.5
    assert np.max(np.abs(np.sum(q.phi * data, axis=1) - (g @ x + 2.5))) < 1e-12


def test_basis_size_is_checked():
    with pytest.raises(ValueError):
        oracle.basis_values(np.zeros(3), 7)
