"""Quadratic MLS basis (m = 10) through the C ABI against the oracle.

Section 2 leaves the basis size m free (Pascal's pyramid; the paper runs
m = 4 and notes that fast-MLS does not depend on m).  With basis = 10 the
exact build solves a 10x10 moment system per marker, and the fast-MLS table
holds quadratic exact shape functions.  Shape functions, c_l, interpolation
and spreading are compared element by element with the oracle at the same
tolerances as the linear basis (double 1e-12, single 1e-5; the quadratic A is
well conditioned, cond_1 about 30 on these grids), plus the quadratic
reproduction the basis guarantees.  Calls the basis does not support are
refused.
"""

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import DEV, fast_tie_fix, home_linear, normwise, run_gpu, run_oracle
from workloads import make_workload
from workloads.fields import field_full_np

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_01113_gb300 import api as _api
    torch.cuda.set_device(0)
    return _api


def _compare(g, r, tol, keys=("phi", "c", "U", "f")):
    errs = {k: normwise(g[k], r[k]) for k in keys}
    assert all(e <= tol for e in errs.values()), errs
    return errs


def _quadratic_moments(grid, x, phi):
    """max over markers and the ten monomials q of |sum_k phi_k q(xi_k) - q(0)|, xi in home widths."""
    sup = oracle.support(grid, np.asarray(x, dtype=np.float64))
    xi = np.stack([(sup.pos[d] - x[d][:, None]) / sup.hwidth[d][:, None] for d in range(3)])
    P = oracle.basis_values(xi, 10)                        # (M, 27, 10)
    rep = np.einsum("mk,mki->mi", phi, P)
    rep[:, 0] -= 1.0
    return np.max(np.abs(rep[sup.ok]))


@pytest.mark.parametrize("method", ["exact", "fast"])
def test_single_sphere_f64_quadratic(api, method):
    """One level-4 icosphere (5120 markers) in a periodic 64^3 grid, double precision."""
    w = make_workload("c1")
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices, w.tri, "f64")
    u = field_full_np(w.modes, w.faces)
    F = w.forces()
    ctx = api.Context(w.faces, w.periodic, real="f64", basis=10)
    g = run_gpu(ctx, x, area, method, torch.as_tensor(u, device=DEV), F)
    r = run_oracle(grid, x, area, method, u, F, basis=10)
    assert g["status"]["dropped"] == 0
    assert np.array_equal(g["home"], home_linear(r["tr"].sup, grid.n))
    _compare(g, r, TOL["f64"])
    if method == "exact":
        assert _quadratic_moments(grid, x, g["phi"]) < 1e-12


@pytest.mark.parametrize("method", ["exact", "fast"])
def test_stretched_f32_quadratic(api, method):
    """Deformed bodies in a grid tanh-stretched and walled in z, single precision."""
    w = make_workload("c3", n=96, n_bodies=16)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = field_full_np(w.modes, w.faces, np.float32)
    F = w.forces().astype(np.float32)
    ctx = api.Context(w.faces, w.periodic, real="f32", basis=10)
    g = run_gpu(ctx, x, area, method, torch.as_tensor(u, device=DEV), F)
    r = run_oracle(grid, x, area, method, u, F, basis=10)
    assert g["status"]["dropped"] == 0
    assert np.array_equal(g["home"], home_linear(r["tr"].sup, grid.n))
    if method == "fast":
        resolved, unresolved = fast_tie_fix(grid, x, g["phi"], r["phi"], TOL["f32"], basis=10)
        assert unresolved == 0 and resolved <= max(3, 1e-4 * x.shape[1])
        if resolved == 0:
            _compare(g, r, TOL["f32"], ("c", "U", "f"))
    else:
        _compare(g, r, TOL["f32"])
        assert _quadratic_moments(grid, x, g["phi"]) < 1e-5


def test_quadratic_differs_from_linear(api):
    """The option reaches the kernels: the two bases give different phi on the same markers."""
    w = make_workload("c1")
    x, area = oracle.marker_prep(w.vertices, w.tri, "f64")
    lin = run_gpu(api.Context(w.faces, w.periodic, real="f64"), x, area, "exact")
    quad = run_gpu(api.Context(w.faces, w.periodic, real="f64", basis=10), x, area, "exact")
    assert np.max(np.abs(lin["phi"] - quad["phi"])) > 1e-3


def test_ill_conditioned_quadratic_goes_to_double(api):
    """cond_max below every cond_1(A) sends every single-precision quadratic solve to the double path."""
    w = make_workload("c3", n=96, n_bodies=4)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    ctx = api.Context(w.faces, w.periodic, real="f32", basis=10, cond_max=1.0)
    g = run_gpu(ctx, x, area, "exact")
    r = run_oracle(grid, x, area, "exact", basis=10)
    assert g["status"]["refined_fp64"] == x.shape[1]
    _compare(g, r, TOL["f32"], ("phi", "c"))


def test_unsupported_with_quadratic_basis(api):
    from paper_1805_01113_gb300 import binding as B
    w = make_workload("c1")
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    ctx = api.Context(w.faces, w.periodic, real="f32", basis=10)
    with pytest.raises(B.MlsError) as e:
        ctx.surrogate_params(np.zeros(B.MLS_MLP_PARAMS, dtype=np.float32))
    assert e.value.code == B.MLS_ERR_UNSUPPORTED
    T = ctx.transfer(x.shape[1])
    xt, at = torch.as_tensor(x, device=DEV), torch.as_tensor(area, device=DEV)
    ctx.build_transfer(T, xt, at, "exact")
    u = torch.zeros((3,) + ctx.n[::-1], dtype=torch.float32, device=DEV)
    with pytest.raises(B.MlsError) as e:
        ctx.interpolate_gradient(T, xt, u)
    assert e.value.code == B.MLS_ERR_UNSUPPORTED
    T.close()
