"""mls_build_interpolate (build and interpolation in one call) through the C ABI.

For exact-MLS with the linear basis the interpolation runs inside the build
kernel; its U is checked against the CPU oracle at the path's tolerance
(normwise: double 1e-12, single 1e-5, bfloat16-stored field against the
oracle on the same rounded field), and the transfer it leaves (phi, c, home)
against the one mls_build_transfer leaves, so that a later spread sees the
same functions.  Other methods run the two calls in turn.
"""

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import DEV, gpu_transfer, home_linear, normwise, run_gpu, run_oracle
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


def _fused(ctx, x, area, u, method="exact"):
    M = x.shape[1]
    T = ctx.transfer(max(M, 1))
    xt = torch.as_tensor(np.ascontiguousarray(x), device=DEV)
    at = torch.as_tensor(np.ascontiguousarray(area), device=DEV)
    U = ctx.build_interpolate(T, xt, at, u, method=method)
    out = {"status": ctx.status(T), "U": U.double().cpu().numpy()}
    out["phi"], out["c"], out["home"] = gpu_transfer(ctx, T)
    torch.cuda.synchronize()
    T.close()
    return out


def _check_against_separate(g, s, tol_phi):
    assert np.array_equal(g["home"], s["home"])
    assert normwise(g["phi"], s["phi"]) <= tol_phi
    assert normwise(g["c"], s["c"]) <= tol_phi


@pytest.mark.parametrize("workload", ["uniform", "stretched"])
def test_fused_exact_f32(api, workload):
    """Many bodies over many tiles: U against the oracle, phi against the separate build."""
    w = (make_workload("c2", n=96, n_bodies=40) if workload == "uniform"
         else make_workload("c3", n=96, n_bodies=16))
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = field_full_np(w.modes, w.faces, np.float32)
    ut = torch.as_tensor(u, device=DEV)
    ctx = api.Context(w.faces, w.periodic, real="f32")
    g = _fused(ctx, x, area, ut)
    r = run_oracle(grid, x, area, "exact", u)
    s = run_gpu(ctx, x, area, "exact", ut)
    assert g["status"]["dropped"] == 0
    assert np.array_equal(g["home"], home_linear(r["tr"].sup, grid.n))
    assert normwise(g["U"], r["U"]) <= TOL["f32"]
    assert normwise(g["phi"], r["phi"]) <= TOL["f32"]
    assert normwise(g["U"], s["U"]) <= 1e-6
    _check_against_separate(g, s, 1e-6)


def test_fused_exact_f64(api):
    w = make_workload("c1", n=48, level=3, radius=0.3)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices, w.tri, "f64")
    u = field_full_np(w.modes, w.faces)
    ctx = api.Context(w.faces, w.periodic, real="f64")
    g = _fused(ctx, x, area, torch.as_tensor(u, device=DEV))
    r = run_oracle(grid, x, area, "exact", u)
    assert normwise(g["U"], r["U"]) <= TOL["f64"]
    assert normwise(g["phi"], r["phi"]) <= TOL["f64"]


def test_fused_edge_markers_and_dropped(api):
    """Markers on faces and seams, and dropped ones (walls, NaN, outside): U = 0 for the dropped."""
    n = 24
    rng = np.random.default_rng(1805011131)
    faces = [uniform_faces(n), uniform_faces(n), tanh_faces(n, 1.5)]
    pts = np.empty((3, 700))
    for d in range(3):
        pts[d] = rng.uniform(faces[d][1], faces[d][n - 1], size=700)
    special = np.array([
        (faces[0][3], faces[1][5], faces[2][4]),
        (faces[0][0], faces[1][0], faces[2][2]),
        (0.1, 0.2, 0.5 * (faces[2][0] + faces[2][1])),
        (np.nan, 0.0, 0.0),
        (-1.5, 0.0, 0.0),
    ]).T
    x = np.concatenate([pts, special], axis=1).astype(np.float32)
    area = (rng.uniform(0.5, 1.5, size=x.shape[1]) * (2.0 / n) ** 2).astype(np.float32)
    grid = oracle.Grid(faces, (True, True, False))
    u = rng.standard_normal((3, n, n, n)).astype(np.float32)
    ctx = api.Context(faces, (True, True, False), real="f32")
    g = _fused(ctx, x, area, torch.as_tensor(u, device=DEV))
    r = run_oracle(grid, x, area, "exact", u)
    assert g["status"]["dropped"] == 3
    assert np.all(g["U"][:, -3:] == 0.0)
    assert normwise(g["U"], r["U"]) <= TOL["f32"]


def test_fused_double_resolve(api):
    """cond_max = 1 sends every marker to the double re-solve, which interpolates too."""
    w = make_workload("c2", n=64, n_bodies=6)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = field_full_np(w.modes, w.faces, np.float32)
    ctx = api.Context(w.faces, w.periodic, real="f32", cond_max=1.0)
    g = _fused(ctx, x, area, torch.as_tensor(u, device=DEV))
    r = run_oracle(grid, x, area, "exact", u)
    assert g["status"]["refined_fp64"] == x.shape[1]
    assert normwise(g["U"], r["U"]) <= TOL["f32"]


def test_fused_bf16_field(api):
    """bfloat16 field storage: U against the oracle on the same rounded field."""
    w = make_workload("c2", n=64, n_bodies=12)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    ub = torch.as_tensor(field_full_np(w.modes, w.faces, np.float32), device=DEV).to(torch.bfloat16)
    ctx = api.Context(w.faces, w.periodic, real="f32", field="bf16")
    g = _fused(ctx, x, area, ub)
    r = run_oracle(grid, x, area, "exact", ub.double().cpu().numpy())
    assert normwise(g["U"], r["U"]) <= TOL["f32"]


def test_fused_quadratic_runs_both_calls(api):
    """The quadratic exact basis: the call equals build_transfer + interpolate."""
    w = make_workload("c2", n=64, n_bodies=8)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    ut = torch.as_tensor(field_full_np(w.modes, w.faces, np.float32), device=DEV)
    ctx = api.Context(w.faces, w.periodic, real="f32", basis=10)
    g = _fused(ctx, x, area, ut, method="exact")
    s = run_gpu(ctx, x, area, "exact", ut)
    assert np.array_equal(g["U"], s["U"])
    _check_against_separate(g, s, 0.0)


@pytest.mark.parametrize("case", ["uniform", "stretched", "bf16", "f64", "quadratic"])
def test_fused_fast(api, case):
    """Fast-MLS (table in shared memory on the uniform grid, read through the cache on the
    stretched one) runs the two calls in turn: the same transfer and U."""
    if case == "f64":
        w = make_workload("c1", n=32, level=3, radius=0.3)
        x, area = oracle.marker_prep(w.vertices, w.tri, "f64")
        ut = torch.as_tensor(field_full_np(w.modes, w.faces), device=DEV)
        ctx = api.Context(w.faces, w.periodic, real="f64")
    else:
        w = make_workload("c3", n=96, n_bodies=16) if case == "stretched" else make_workload("c2", n=64, n_bodies=12)
        x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
        ut = torch.as_tensor(field_full_np(w.modes, w.faces, np.float32), device=DEV)
        if case == "bf16":
            ut = ut.to(torch.bfloat16)
        ctx = api.Context(w.faces, w.periodic, real="f32", field="bf16" if case == "bf16" else "f32",
                          basis=10 if case == "quadratic" else 4)
    g = _fused(ctx, x, area, ut, method="fast")
    s = run_gpu(ctx, x, area, "fast", ut)
    assert g["status"]["dropped"] == 0
    assert np.array_equal(g["U"], s["U"])
    _check_against_separate(g, s, 0.0)


def test_fused_empty(api):
    w = make_workload("c2", n=64, n_bodies=1)
    ctx = api.Context(w.faces, w.periodic, real="f32")
    T = ctx.transfer(4)
    x = torch.zeros((3, 0), dtype=torch.float32, device=DEV)
    a = torch.zeros((0,), dtype=torch.float32, device=DEV)
    u = torch.zeros((3, 64, 64, 64), dtype=torch.float32, device=DEV)
    U = ctx.build_interpolate(T, x, a, u)
    torch.cuda.synchronize()
    assert U.shape == (3, 0)
    T.close()
