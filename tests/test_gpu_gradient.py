"""Gradient interpolation (mls_interpolate_gradient) against the CPU oracle.

G[c, d, l] = sum_k d_d phi_k^l u_c,k with the derivatives of the exact-MLS
shape functions.  Tolerances are normwise over the whole G array: double
1e-12, single 1e-5.
"""

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import DEV, NP_DT, normwise
from workloads import make_workload, tanh_faces, uniform_faces
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


def _gpu(ctx, x, area, u, method="exact"):
    M = x.shape[1]
    T = ctx.transfer(M)
    xt = torch.as_tensor(np.ascontiguousarray(x), device=DEV)
    ctx.build_transfer(T, xt, torch.as_tensor(np.ascontiguousarray(area), device=DEV), method)
    ut = u if isinstance(u, torch.Tensor) else torch.as_tensor(u, device=DEV)
    G = ctx.interpolate_gradient(T, xt, ut)
    torch.cuda.synchronize()
    return G.double().cpu().numpy()


def _oracle(grid, x, u):
    x64 = np.asarray(x, dtype=np.float64)
    dphi = oracle.shape_exact_gradient(grid, x64, 1.0)
    sup = oracle.support(grid, x64)
    return oracle.interpolate_gradient(dphi, sup, np.asarray(u, dtype=np.float64))


def test_single_sphere_f64(api):
    w = make_workload("c1")
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices, w.tri, "f64")
    u = field_full_np(w.modes, w.faces)
    ctx = api.Context(w.faces, w.periodic, real="f64")
    assert normwise(_gpu(ctx, x, area, u), _oracle(grid, x, u)) <= TOL["f64"]


@pytest.mark.parametrize("real", ["f64", "f32"])
def test_stretched_multibody(api, real):
    w = make_workload("c3", n=64, n_bodies=8)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(NP_DT[real]), w.tri, real)
    u = field_full_np(w.modes, w.faces, NP_DT[real])
    ctx = api.Context(w.faces, w.periodic, real=real)
    G = _gpu(ctx, x, area, u)
    R = _oracle(grid, x, u)
    assert normwise(G, R) <= TOL[real]


def test_linear_field_gives_its_gradient(api):
    """A linear velocity field has a constant gradient, reproduced exactly by
    exact-MLS derivatives away from periodic seams."""
    n = 24
    faces = [uniform_faces(n), uniform_faces(n), tanh_faces(n, 1.5)]
    grid = oracle.Grid(faces, (True, True, False))
    rng = np.random.default_rng(9)
    x = np.stack([rng.uniform(-0.7, 0.7, 2000) for _ in range(3)])
    Bm = rng.normal(size=(3, 3))
    zc, yc, xc = grid.centres[2], grid.centres[1], grid.centres[0]
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    u = np.stack([Bm[c, 0] * X + Bm[c, 1] * Y + Bm[c, 2] * Z for c in range(3)])
    ctx = api.Context(faces, (True, True, False), real="f64")
    G = _gpu(ctx, x, np.full(2000, 1e-4), u)
    assert np.max(np.abs(G - Bm[:, :, None])) < 1e-10


def test_dropped_markers_and_bf16(api):
    faces = [uniform_faces(16), uniform_faces(16), tanh_faces(16, 1.5)]
    grid = oracle.Grid(faces, (True, True, False))
    rng = np.random.default_rng(10)
    x = np.stack([rng.uniform(-0.8, 0.8, 600) for _ in range(3)]).astype(np.float32)
    x[2, :10] = -0.999                                       # wall cell: dropped
    area = np.full(600, 1e-3, dtype=np.float32)
    u = rng.normal(size=(3, 16, 16, 16)).astype(np.float32)
    ub = torch.as_tensor(u, device=DEV).to(torch.bfloat16)
    ctx = api.Context(faces, (True, True, False), real="f32", field="bf16")
    G = _gpu(ctx, x, area, ub)
    assert np.all(G[:, :, :10] == 0)
    R = _oracle(grid, x, ub.double().cpu().numpy())
    assert normwise(G, R) <= TOL["f32"]
