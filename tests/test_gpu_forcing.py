"""Fused direct-forcing transfer (mls_direct_forcing) against the CPU oracle.

U = Phi^T u, F = (V_b - U)/dt, f += sum c phi F (text after Eq. 6 and Eq. 7).
Tolerances are normwise as in the other parity tests: double 1e-12, single
1e-5, bfloat16-stored spread field 1e-2.  V_b is drawn independently of u, so
F is O(1/dt) and its error is that of U scaled by 1/dt.
"""

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import DEV, NP_DT, normwise, run_oracle
from workloads import make_workload, tanh_faces, uniform_faces
from workloads.fields import field_full_np

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
DT = 1e-2


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_01113_gb300 import api as _api
    torch.cuda.set_device(0)
    return _api


def _run(api, ctx, x, area, u, Vb, want_U=True, method="exact"):
    M = x.shape[1]
    T = ctx.transfer(max(M, 1))
    ctx.build_transfer(T, torch.as_tensor(np.ascontiguousarray(x), device=DEV),
                       torch.as_tensor(np.ascontiguousarray(area), device=DEV), method)
    ut = u if isinstance(u, torch.Tensor) else torch.as_tensor(u, device=DEV)
    f = torch.zeros((3,) + ctx.n[::-1], dtype=ctx.field_t, device=DEV)
    U = torch.full((3, M), 7.0, dtype=ctx.real_t, device=DEV) if want_U else None
    F, U = ctx.direct_forcing(T, ut, torch.as_tensor(np.ascontiguousarray(Vb), device=DEV), DT, f, U=U)
    torch.cuda.synchronize()
    out = {"F": F.double().cpu().numpy(), "f": f.double().cpu().numpy(), "status": ctx.status(T), "T": T}
    if U is not None:
        out["U"] = U.double().cpu().numpy()
    return out


def _oracle(grid, x, area, u, Vb, method="exact"):
    r = run_oracle(grid, x, area, method)
    U, F, sp = oracle.direct_forcing(r["tr"], r["c"], np.asarray(u, dtype=np.float64), Vb, DT, grid.n)
    return {"U": U, "F": F, "f": sp.to_dense(grid.n), "tr": r["tr"]}


def _check(g, r, tol, keys=("U", "F", "f")):
    errs = {k: normwise(g[k], r[k]) for k in keys if k in g}
    assert all(e <= tol for e in errs.values()), errs


def test_single_sphere_f64(api):
    """Double precision (the composed path), one level-4 icosphere in 64^3."""
    w = make_workload("c1")
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices, w.tri, "f64")
    u = field_full_np(w.modes, w.faces)
    Vb = np.random.default_rng(3).normal(size=x.shape)
    ctx = api.Context(w.faces, w.periodic, real="f64")
    g = _run(api, ctx, x, area, u, Vb)
    r = _oracle(grid, x, area, u, Vb)
    _check(g, r, TOL["f64"])


@pytest.mark.parametrize("brick", [(3, 3, 3), (3, 3, 2), (4, 4, 2)])
def test_multibody_f32(api, brick):
    """Single precision, fused kernel (vector flush), several tile shapes."""
    w = make_workload("c2", n=64, n_bodies=12)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = field_full_np(w.modes, w.faces, np.float32)
    Vb = np.random.default_rng(4).normal(size=x.shape).astype(np.float32)
    ctx = api.Context(w.faces, w.periodic, real="f32", brick_log2=brick)
    g = _run(api, ctx, x, area, u, Vb)
    r = _oracle(grid, x, area, u, Vb)
    assert g["status"]["dropped"] == 0
    _check(g, r, TOL["f32"])


def test_fused_matches_separate_calls(api):
    """The fused pass equals interpolate -> (Vb - U)/dt -> spread on the same transfer."""
    w = make_workload("c2", n=64, n_bodies=10)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = torch.as_tensor(field_full_np(w.modes, w.faces, np.float32), device=DEV)
    Vb = torch.as_tensor(np.random.default_rng(5).normal(size=x.shape).astype(np.float32), device=DEV)
    ctx = api.Context(w.faces, w.periodic, real="f32")
    g = _run(api, ctx, x, area, u, Vb.cpu().numpy())
    U2 = ctx.interpolate(g["T"], u)
    F2 = (Vb - U2) / DT
    f2 = torch.zeros_like(u)
    ctx.spread(g["T"], F2, f2)
    torch.cuda.synchronize()
    assert np.array_equal(g["U"], U2.double().cpu().numpy())
    assert normwise(g["F"], F2.double().cpu().numpy()) <= 1e-6
    assert normwise(g["f"], f2.double().cpu().numpy()) <= 1e-5


def test_without_U_output(api):
    w = make_workload("c2", n=64, n_bodies=6)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = field_full_np(w.modes, w.faces, np.float32)
    Vb = np.random.default_rng(6).normal(size=x.shape).astype(np.float32)
    ctx = api.Context(w.faces, w.periodic, real="f32")
    g = _run(api, ctx, x, area, u, Vb, want_U=False)
    assert "U" not in g
    r = _oracle(grid, x, area, u, Vb)
    _check(g, r, TOL["f32"], ("F", "f"))


@pytest.mark.parametrize("real", ["f64", "f32"])
def test_edge_and_dropped_markers(api, real):
    """Periodic seams, a stretched non-periodic axis, odd x extent (scalar flush)
    and markers without support (U = F = 0, no field)."""
    rng = np.random.default_rng(11)
    n = 15
    faces = [uniform_faces(n), uniform_faces(16), tanh_faces(12, 1.5)]
    periodic = (True, True, False)
    grid = oracle.Grid(faces, periodic)
    M = 3000
    x = np.empty((3, M))
    x[0] = rng.uniform(-1, 1, M)
    x[1] = rng.uniform(-1, 1, M)
    x[2] = rng.uniform(faces[2][1], faces[2][11], M)
    x[0, :100] = rng.uniform(faces[0][0], faces[0][1], 100)     # home cell x = 0 (seam)
    x[2, 100:150] = 0.5 * (faces[2][0] + faces[2][1])          # wall cell: dropped
    x[0, 150] = np.nan                                          # non-finite: dropped
    x = x.astype(NP_DT[real])
    area = (rng.uniform(0.5, 1.5, M) * (2.0 / n) ** 2).astype(NP_DT[real])
    u = rng.normal(size=(3, 12, 16, n)).astype(NP_DT[real])
    Vb = rng.normal(size=(3, M)).astype(NP_DT[real])
    ctx = api.Context(faces, periodic, real=real, brick_log2=(2, 2, 2))
    g = _run(api, ctx, x, area, u, Vb)
    r = _oracle(grid, x, area, u, Vb)
    dropped = ~r["tr"].sup.ok
    assert dropped.sum() == 51 and g["status"]["dropped"] == 51
    assert np.all(g["U"][:, dropped] == 0) and np.all(g["F"][:, dropped] == 0)
    _check(g, r, TOL[real])


def test_bf16_fields(api):
    """bfloat16 u and f: U and F at single-precision accuracy from identical inputs,
    the spread field within the stated bf16 bound."""
    w = make_workload("c2", n=64, n_bodies=12)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = torch.as_tensor(field_full_np(w.modes, w.faces), device=DEV).to(torch.bfloat16)
    Vb = np.random.default_rng(8).normal(size=x.shape).astype(np.float32)
    ctx = api.Context(w.faces, w.periodic, real="f32", field="bf16")
    g = _run(api, ctx, x, area, u, Vb)
    r = _oracle(grid, x, area, u.double().cpu().numpy(), Vb)
    _check(g, r, TOL["f32"], ("U", "F"))
    assert normwise(g["f"], r["f"]) <= 1e-2


def test_invalid_dt(api):
    from paper_1805_01113_gb300 import binding as B
    faces = [uniform_faces(8)] * 3
    ctx = api.Context(faces, (True, True, True), real="f32")
    T = ctx.transfer(4)
    x = torch.zeros((3, 4), dtype=torch.float32, device=DEV)
    ctx.build_transfer(T, x, torch.full((4,), 1e-3, dtype=torch.float32, device=DEV))
    u = torch.zeros((3, 8, 8, 8), dtype=torch.float32, device=DEV)
    for dt in (0.0, -1.0, float("nan")):
        with pytest.raises(B.MlsError) as e:
            ctx.direct_forcing(T, u, torch.zeros((3, 4), dtype=torch.float32, device=DEV), dt, torch.zeros_like(u))
        assert e.value.code == B.MLS_ERR_INVALID_ARG


# ---- mls_build_direct_forcing: the build and the direct forcing in one call


def _run_built(api, ctx, x, area, u, Vb, want_U=True, method="exact"):
    M = x.shape[1]
    T = ctx.transfer(max(M, 1))
    ut = u if isinstance(u, torch.Tensor) else torch.as_tensor(u, device=DEV)
    f = torch.zeros((3,) + ctx.n[::-1], dtype=ctx.field_t, device=DEV)
    U = torch.full((3, M), 7.0, dtype=ctx.real_t, device=DEV) if want_U else None
    F, U = ctx.build_direct_forcing(T, torch.as_tensor(np.ascontiguousarray(x), device=DEV),
                                    torch.as_tensor(np.ascontiguousarray(area), device=DEV), ut,
                                    torch.as_tensor(np.ascontiguousarray(Vb), device=DEV), DT, f, U=U,
                                    method=method)
    torch.cuda.synchronize()
    out = {"F": F.double().cpu().numpy(), "f": f.double().cpu().numpy(), "status": ctx.status(T), "T": T}
    if U is not None:
        out["U"] = U.double().cpu().numpy()
    return out


@pytest.mark.parametrize("want_U", [True, False])
@pytest.mark.parametrize("workload", ["uniform", "stretched"])
def test_build_direct_forcing_f32(api, workload, want_U):
    w = (make_workload("c2", n=64, n_bodies=12) if workload == "uniform"
         else make_workload("c3", n=96, n_bodies=16))
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = field_full_np(w.modes, w.faces, np.float32)
    Vb = np.random.default_rng(12).normal(size=x.shape).astype(np.float32)
    ctx = api.Context(w.faces, w.periodic, real="f32")
    g = _run_built(api, ctx, x, area, u, Vb, want_U=want_U)
    r = _oracle(grid, x, area, u, Vb)
    assert g["status"]["dropped"] == 0
    assert ("U" in g) == want_U
    _check(g, r, TOL["f32"])
    # the same as the two calls on the transfer this call built
    s = _run(api, ctx, x, area, u, Vb)
    assert normwise(g["F"], s["F"]) <= 1e-6 and normwise(g["f"], s["f"]) <= 1e-5


@pytest.mark.parametrize("real", ["f64", "f32"])
def test_build_direct_forcing_edges(api, real):
    """Seams, a stretched walled axis, odd x extent, dropped markers (U = F = 0), and
    cond_max = 1 in single precision (every marker through the double re-solve)."""
    rng = np.random.default_rng(13)
    n = 15
    faces = [uniform_faces(n), uniform_faces(16), tanh_faces(12, 1.5)]
    periodic = (True, True, False)
    grid = oracle.Grid(faces, periodic)
    M = 3000
    x = np.empty((3, M))
    x[0] = rng.uniform(-1, 1, M)
    x[1] = rng.uniform(-1, 1, M)
    x[2] = rng.uniform(faces[2][1], faces[2][11], M)
    x[0, :100] = rng.uniform(faces[0][0], faces[0][1], 100)
    x[2, 100:150] = 0.5 * (faces[2][0] + faces[2][1])
    x[0, 150] = np.nan
    x = x.astype(NP_DT[real])
    area = (rng.uniform(0.5, 1.5, M) * (2.0 / n) ** 2).astype(NP_DT[real])
    u = rng.normal(size=(3, 12, 16, n)).astype(NP_DT[real])
    Vb = rng.normal(size=(3, M)).astype(NP_DT[real])
    for cond_max in ((1e6, 1.0) if real == "f32" else (1e6,)):
        ctx = api.Context(faces, periodic, real=real, brick_log2=(2, 2, 2), cond_max=cond_max)
        g = _run_built(api, ctx, x, area, u, Vb)
        r = _oracle(grid, x, area, u, Vb)
        dropped = ~r["tr"].sup.ok
        assert g["status"]["dropped"] == 51
        if cond_max == 1.0:
            assert g["status"]["refined_fp64"] == M - 51
        assert np.all(g["U"][:, dropped] == 0) and np.all(g["F"][:, dropped] == 0)
        _check(g, r, TOL[real])


def test_build_direct_forcing_fast_and_invalid_dt(api):
    """Fast-MLS runs the two calls in turn; dt must be positive and finite."""
    from paper_1805_01113_gb300 import binding as B
    w = make_workload("c2", n=64, n_bodies=6)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = field_full_np(w.modes, w.faces, np.float32)
    Vb = np.random.default_rng(14).normal(size=x.shape).astype(np.float32)
    ctx = api.Context(w.faces, w.periodic, real="f32")
    g = _run_built(api, ctx, x, area, u, Vb, method="fast")
    s = _run(api, ctx, x, area, u, Vb, method="fast")
    assert np.array_equal(g["F"], s["F"]) and np.array_equal(g["U"], s["U"])
    T = ctx.transfer(x.shape[1])
    ut = torch.as_tensor(u, device=DEV)
    for dt in (0.0, -1.0, float("nan")):
        with pytest.raises(B.MlsError) as e:
            ctx.build_direct_forcing(T, torch.as_tensor(x, device=DEV), torch.as_tensor(area, device=DEV), ut,
                                     torch.as_tensor(Vb, device=DEV), dt, torch.zeros_like(ut))
        assert e.value.code == B.MLS_ERR_INVALID_ARG
