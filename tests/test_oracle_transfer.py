"""Pins for interpolation, spreading and the scaling factor c_l (Section 2, Eqs. 7-8)."""

import numpy as np
import pytest

import oracle
from workloads import uniform_faces, tanh_faces

RNG = np.random.default_rng(21)


def _grids():
    yield "uniform", oracle.Grid([uniform_faces(12)] * 3, (True, True, True))
    yield "stretched", oracle.Grid([uniform_faces(12), uniform_faces(14), tanh_faces(16, 1.5)],
                                   (True, True, False))


def _markers(grid, m, interior=2):
    x = np.empty((3, m))
    for d in range(3):
        f = grid.faces[d]
        x[d] = RNG.uniform(f[interior], f[grid.n[d] - interior], size=m)
    return x


def _field(grid, fn):
    zc, yc, xc = (grid.centres[2], grid.centres[1], grid.centres[0])
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    return fn(X, Y, Z)


@pytest.mark.parametrize("method", ["exact", "fast"])
def test_interp_constant_and_linear(method):
    for _, grid in _grids():
        x = _markers(grid, 150)
        tr = (oracle.shape_exact(grid, x, 1.0) if method == "exact"
              else oracle.shape_fast(grid, x, 1.0, 9))
        const = np.stack([_field(grid, lambda X, Y, Z: 0 * X + v) for v in (1.0, -2.0, 0.5)])
        U = oracle.interpolate(tr, const)
        assert np.max(np.abs(U - np.array([1.0, -2.0, 0.5])[:, None])) < 1e-13
        if method == "exact":
            # Linear fields are reproduced exactly (linear basis, m = 4); the
            # markers stay away from periodic seams so the field is single-valued.
            B = RNG.normal(size=(3, 3))
            a = RNG.normal(size=3)
            lin = np.stack([_field(grid, lambda X, Y, Z, c=c: a[c] + B[c, 0] * X + B[c, 1] * Y + B[c, 2] * Z)
                            for c in range(3)])
            U = oracle.interpolate(tr, lin)
            ref = a[:, None] + B @ x
            assert np.max(np.abs(U - ref)) < 1e-12


def test_scaling_factor_uniform_closed_form():
    """On a uniform grid h_l = h and sum_k phi_k dV_k = h^3, so c_l = A_l / h^2 (Eq. 8)."""
    grid = oracle.Grid([uniform_faces(10)] * 3, (True, True, True))
    h = 0.2
    x = _markers(grid, 100, interior=0)
    area = RNG.uniform(0.1, 2.0, size=100) * h * h
    for tr in (oracle.shape_exact(grid, x, 1.0), oracle.shape_fast(grid, x, 1.0, 9)):
        c = oracle.forcing_scale(tr, area)
        assert np.max(np.abs(c - area / h ** 2)) < 1e-12


@pytest.mark.parametrize("method", ["exact", "fast"])
def test_conservation_eq7(method):
    """sum_k f_k dV_k = sum_l F_l dV_l (Eq. 7); with dV_l = A_l h on a uniform grid."""
    n = 10
    grid = oracle.Grid([uniform_faces(n)] * 3, (True, True, True))
    h = 2.0 / n
    m = 300
    x = _markers(grid, m, interior=0)
    area = RNG.uniform(0.2, 1.0, size=m) * h * h
    F = RNG.normal(size=(3, m))
    tr = oracle.shape_exact(grid, x, 1.0) if method == "exact" else oracle.shape_fast(grid, x, 1.0, 9)
    c = oracle.forcing_scale(tr, area)
    f = oracle.spread(tr, c, F, grid.n).to_dense(grid.n)
    lhs = f.reshape(3, -1).sum(1) * h ** 3
    rhs = (F * area * h).sum(1)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(rhs)) + 1e-15


@pytest.mark.parametrize("method", ["exact", "fast"])
def test_adjointness(method):
    """<interp(u), c F>_markers = <u, spread(F)>_cells for any u, F."""
    for _, grid in _grids():
        m = 200
        x = _markers(grid, m, interior=1)
        tr = oracle.shape_exact(grid, x, 1.0) if method == "exact" else oracle.shape_fast(grid, x, 1.0, 9)
        area = RNG.uniform(0.5, 1.5, size=m) * 1e-2
        c = oracle.forcing_scale(tr, area)
        u = RNG.normal(size=(3,) + grid.n[::-1])
        F = RNG.normal(size=(3, m))
        U = oracle.interpolate(tr, u)
        f = oracle.spread(tr, c, F, grid.n).to_dense(grid.n)
        lhs = np.sum(U * c * F)
        rhs = np.sum(u * f)
        assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1.0)


def test_spread_single_marker():
    """One marker: f_k = c phi_k F, its total is c F (partition of unity)."""
    grid = oracle.Grid([uniform_faces(8)] * 3, (True, True, True))
    x = np.array([[0.013], [-0.41], [0.77]])
    tr = oracle.shape_exact(grid, x, 1.0)
    c = np.array([2.5])
    F = np.array([[1.0], [-3.0], [0.25]])
    sp = oracle.spread(tr, c, F, grid.n)
    assert len(sp.keys) == 27
    assert np.max(np.abs(sp.values.sum(1) - 2.5 * F[:, 0])) < 1e-14


def test_unusable_markers_contribute_nothing():
    grid = oracle.Grid([uniform_faces(8)] * 3, (True, True, False))
    x = np.array([[0.1, 0.1], [0.2, 0.2], [0.0, -0.99]])     # second marker in wall cell 0
    tr = oracle.shape_exact(grid, x, 1.0)
    assert list(tr.sup.ok) == [True, False]
    assert np.all(tr.phi[1] == 0)
    c = oracle.forcing_scale(tr, np.array([0.01, 0.01]))
    assert c[1] == 0
    sp = oracle.spread(tr, c, np.ones((3, 2)), grid.n)
    assert len(sp.keys) == 27


# ---- direct forcing (text after Eq. 6 and Eq. 7) --------------------------------

@pytest.mark.parametrize("method", ["exact", "fast"])
def test_direct_forcing_linear_field_recovers_force(method):
    """On a linear velocity field, exact-MLS interpolation is exact, so with
    V_b = u(x_l) + dt G_l the force is G_l; fast-MLS is exact on constants."""
    for _, grid in _grids():
        m = 120
        x = _markers(grid, m)
        tr = oracle.shape_exact(grid, x, 1.0) if method == "exact" else oracle.shape_fast(grid, x, 1.0, 9)
        a = np.array([0.3, -1.1, 2.0])
        B = RNG.normal(size=(3, 3)) if method == "exact" else np.zeros((3, 3))
        u = np.stack([_field(grid, lambda X, Y, Z, i=i: a[i] + B[i, 0] * X + B[i, 1] * Y + B[i, 2] * Z)
                      for i in range(3)])
        dt = 2.5e-3
        G = RNG.normal(size=(3, m))
        Vb = a[:, None] + B @ x + dt * G
        c = oracle.forcing_scale(tr, np.full(m, 1e-3))
        U, F, _ = oracle.direct_forcing(tr, c, u, Vb, dt, grid.n)
        assert np.max(np.abs(U - (a[:, None] + B @ x))) < 1e-12
        assert np.max(np.abs(F - G)) < 1e-8            # (V_b - U)/dt: rounding of U amplified by 1/dt


def test_direct_forcing_at_target_is_zero():
    """V_b equal to the interpolated velocity gives no force and no field."""
    grid = oracle.Grid([uniform_faces(10)] * 3, (True, True, True))
    x = _markers(grid, 80, interior=0)
    tr = oracle.shape_exact(grid, x, 1.0)
    u = RNG.normal(size=(3,) + grid.n[::-1])
    Vb = oracle.interpolate(tr, u)
    c = oracle.forcing_scale(tr, np.full(80, 1e-3))
    U, F, f = oracle.direct_forcing(tr, c, u, Vb, 0.01, grid.n)
    assert np.array_equal(U, Vb) and np.all(F == 0) and np.all(f.values == 0)


def test_direct_forcing_conserves_momentum_and_drops():
    """sum_k f_k dV_k = sum_l F_l dV_l (Eq. 7) for the computed forces; a marker
    without support gets U = F = 0 and adds nothing."""
    n = 10
    grid = oracle.Grid([uniform_faces(n)] * 3, (True, True, False))
    h = 2.0 / n
    x = _markers(grid, 200, interior=1)
    x[:, -1] = [0.1, 0.2, -0.99]                       # wall cell z = 0: no support
    area = RNG.uniform(0.2, 1.0, size=200) * h * h
    tr = oracle.shape_exact(grid, x, 1.0)
    assert not tr.sup.ok[-1] and tr.sup.ok[:-1].all()
    c = oracle.forcing_scale(tr, area)
    u = RNG.normal(size=(3,) + grid.n[::-1])
    Vb = RNG.normal(size=(3, 200))
    U, F, sp = oracle.direct_forcing(tr, c, u, Vb, 0.05, grid.n)
    assert np.all(U[:, -1] == 0) and np.all(F[:, -1] == 0)
    assert np.max(np.abs(F[:, :-1] - (Vb[:, :-1] - U[:, :-1]) / 0.05)) < 1e-12
    f = sp.to_dense(grid.n)
    lhs = f.reshape(3, -1).sum(1) * h ** 3
    rhs = (F * area * h).sum(1)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(rhs))


def test_quadratic_basis_interpolates_quadratic_fields():
    """With m = 10 the interpolation U = Phi^T u reproduces every quadratic field
    exactly (the linear basis does not), and the scaling factor and Eq. 7
    conservation are unchanged, since they rest only on the partition of unity."""
    for _, grid in _grids():
        x = _markers(grid, 150)
        q = oracle.shape_exact(grid, x, 1.0, basis=10)
        lin = oracle.shape_exact(grid, x, 1.0, basis=4)
        C = RNG.normal(size=(3, 10))
        mono = lambda X, Y, Z: [np.ones_like(X), X, Y, Z, X * X, Y * Y, Z * Z, X * Y, Y * Z, Z * X]
        field = np.stack([_field(grid, lambda X, Y, Z, c=c: sum(C[c, i] * t for i, t in enumerate(mono(X, Y, Z))))
                          for c in range(3)])
        ref = np.stack([sum(C[c, i] * t for i, t in enumerate(mono(x[0], x[1], x[2]))) for c in range(3)])
        assert np.max(np.abs(oracle.interpolate(q, field) - ref)) < 1e-11 * np.max(np.abs(ref))
        assert np.max(np.abs(oracle.interpolate(lin, field) - ref)) > 1e-4 * np.max(np.abs(ref))
    n = 10
    grid = oracle.Grid([uniform_faces(n)] * 3, (True, True, True))
    h = 2.0 / n
    m = 200
    x = _markers(grid, m, interior=0)
    area = RNG.uniform(0.2, 1.0, size=m) * h * h
    tr = oracle.shape_exact(grid, x, 1.0, basis=10)
    c = oracle.forcing_scale(tr, area)
    assert np.max(np.abs(c - area / h ** 2)) < 1e-12
    F = RNG.normal(size=(3, m))
    f = oracle.spread(tr, c, F, grid.n).to_dense(grid.n)
    assert np.max(np.abs(f.reshape(3, -1).sum(1) * h ** 3 - (F * area * h).sum(1))) < 1e-12
