"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerances (normwise, max|gpu - oracle| / max|oracle| per output array):
double 1e-12, single 1e-5, bfloat16-stored spread field 1e-2.  Sizes span
many spreading tiles and blocks with ragged tails; the full-size multi-body
case runs in the launch configuration the benchmark times and is checked on
sampled markers and cells plus conservation and adjointness.
"""

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import DEV, NP_DT, fast_tie_fix, home_linear, normwise, oracle_outputs_with_phi, run_gpu, run_oracle
from workloads import make_workload, tanh_faces, uniform_faces
from workloads.fields import field_full_np, field_full_torch

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
    errs = {k: normwise(g[k], r[k]) for k in keys if k in g and k in r}
    assert all(e <= tol for e in errs.values()), errs
    return errs


@pytest.mark.parametrize("real", ["f64", "f32"])
def test_marker_prep_bit_exact(api, real):
    w = make_workload("c2", n=128, n_bodies=40)
    ctx = api.Context(w.faces, w.periodic, real=real)
    V = w.vertices.astype(NP_DT[real])
    tri = w.tri.copy()
    tri[5] = [0, 1, len(V)]                                # out-of-range vertex index
    x, a = ctx.marker_prep(torch.as_tensor(V, device=DEV), torch.as_tensor(tri, device=DEV))
    xr, ar = oracle.marker_prep(V, np.where(tri < len(V), tri, 0), real)
    xg, ag = x.cpu().numpy(), a.cpu().numpy()
    good = np.ones(len(tri), bool)
    good[5] = False
    assert np.isnan(xg[:, 5]).all() and np.isnan(ag[5])
    assert np.array_equal(xg[:, good], xr[:, good])
    assert np.array_equal(ag[good], ar[good])


@pytest.mark.parametrize("real", ["f64", "f32"])
def test_marker_prep_in_pieces(api, real):
    """Markers prepared body range by body range, each range after its own
    vertices are copied (the rest of the vertex array still garbage), equal
    the whole-array preparation bit for bit; bad ranges are refused."""
    from paper_1805_01113_gb300 import binding as B
    w = make_workload("c2", n=128, n_bodies=40)
    ctx = api.Context(w.faces, w.periodic, real=real)
    V = torch.as_tensor(w.vertices.astype(NP_DT[real]), device=DEV)
    tri = torch.as_tensor(w.tri, device=DEV)
    x0, a0 = ctx.marker_prep(V, tri)
    nt = tri.shape[0]
    Vp = torch.full_like(V, float("nan"))
    x = torch.full((3, nt), -7.0, dtype=V.dtype, device=DEV)
    a = torch.full((nt,), -7.0, dtype=V.dtype, device=DEV)
    nb = len(w.body_faces) - 1
    cuts = [int(w.body_faces[b]) for b in (0, 7, 8, 23, nb)]      # 7..8: a range of one body
    for t0, t1 in zip(cuts[:-1], cuts[1:]):
        v1 = int(w.tri[:t1].max()) + 1
        Vp[:v1] = V[:v1]
        ctx.marker_prep(Vp, tri, x, a, begin=t0, end=t1)
        assert bool((x[:, t1:] == -7.0).all()) and bool((a[t1:] == -7.0).all())
    ctx.marker_prep(Vp, tri, x, a, begin=nt, end=nt)                 # empty range: nothing to do
    assert torch.equal(x, x0) and torch.equal(a, a0)
    for t0, t1 in ((-1, 5), (6, 5), (0, nt + 1)):
        with pytest.raises(B.MlsError) as e:
            ctx.marker_prep(V, tri, x, a, begin=t0, end=t1)
        assert e.value.code == B.MLS_ERR_INVALID_ARG


@pytest.mark.parametrize("method", ["exact", "fast"])
def test_single_sphere_f64(api, method):
    """One level-4 icosphere (5120 markers) in a periodic 64^3 grid, double precision."""
    w = make_workload("c1")
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices, w.tri, "f64")
    u = field_full_np(w.modes, w.faces)
    F = w.forces()
    ctx = api.Context(w.faces, w.periodic, real="f64")
    g = run_gpu(ctx, x, area, method, torch.as_tensor(u, device=DEV), F)
    r = run_oracle(grid, x, area, method, u, F)
    assert g["status"]["dropped"] == 0
    assert np.array_equal(g["home"], home_linear(r["tr"].sup, grid.n))
    _compare(g, r, TOL["f64"])
    assert np.all(g["f"][r["f"] == 0] == 0)               # untouched cells stay exactly zero


@pytest.mark.parametrize("method", ["exact", "fast"])
def test_multibody_f32(api, method):
    """48 ellipsoids (61440 markers) in a periodic 128^3 grid, single precision."""
    w = make_workload("c2", n=128, n_bodies=48)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = field_full_np(w.modes, w.faces, np.float32)
    F = w.forces().astype(np.float32)
    ctx = api.Context(w.faces, w.periodic, real="f32")
    g = run_gpu(ctx, x, area, method, torch.as_tensor(u, device=DEV), F)
    r = run_oracle(grid, x, area, method, u, F)
    assert g["status"]["dropped"] == 0
    assert np.array_equal(g["home"], home_linear(r["tr"].sup, grid.n))
    if method == "fast":
        fixed = r["phi"].copy()
        _, unresolved = fast_tie_fix(grid, x, g["phi"], r["phi"], TOL["f32"], fixed=fixed)
        assert unresolved == 0
        _compare(g, oracle_outputs_with_phi(grid, r["tr"], fixed, area, u, F), TOL["f32"])
    else:
        _compare(g, r, TOL["f32"])


@pytest.mark.parametrize("method", ["exact", "fast"])
def test_stretched_f32(api, method):
    """Deformed bodies in a grid tanh-stretched and walled in z (one table per z cell for fast-MLS)."""
    w = make_workload("c3", n=96, n_bodies=16)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = field_full_np(w.modes, w.faces, np.float32)
    F = w.forces().astype(np.float32)
    ctx = api.Context(w.faces, w.periodic, real="f32")
    g = run_gpu(ctx, x, area, method, torch.as_tensor(u, device=DEV), F)
    r = run_oracle(grid, x, area, method, u, F)
    assert g["status"]["dropped"] == 0
    assert np.array_equal(g["home"], home_linear(r["tr"].sup, grid.n))
    if method == "fast":
        fixed = r["phi"].copy()
        resolved, unresolved = fast_tie_fix(grid, x, g["phi"], r["phi"], TOL["f32"], fixed=fixed)
        assert unresolved == 0 and resolved <= max(3, 1e-4 * x.shape[1])
        # Every output against the oracle recomputed on the GPU's sub-cell choices.
        rf = oracle_outputs_with_phi(grid, r["tr"], fixed, area, u, F)
        _compare(g, rf, TOL["f32"])
    else:
        _compare(g, r, TOL["f32"])


def _below(v, real):
    """Largest number of the path's precision below v."""
    dt = NP_DT[real]
    return float(np.nextafter(dt(v), dt(-np.inf)))


def _edge_markers(n, rng, real):
    """1000 random markers plus faces, periodic seams, walls, NaN/inf and outside points."""
    faces = [uniform_faces(n), uniform_faces(n), tanh_faces(n, 1.5)]
    x = np.empty((3, 1000))
    for d in range(3):
        x[d] = rng.uniform(faces[d][1], faces[d][n - 1], size=1000)
    special = [
        (faces[0][3], faces[1][5], faces[2][4]),            # exactly on faces: lower cell wins
        (faces[0][0], faces[1][0], faces[2][2]),            # periodic seam at the low end
        (_below(faces[0][n], real), _below(faces[1][n], real), faces[2][n - 2]),  # just below the high end
        (0.1, 0.2, 0.5 * (faces[2][0] + faces[2][1])),     # wall cell z=0: dropped
        (0.1, 0.2, 0.5 * (faces[2][n - 1] + faces[2][n])),  # wall cell z=n-1: dropped
        (np.nan, 0.0, 0.0),                                 # non-finite: dropped
        (1.0, 0.0, 0.0),                                    # x = upper face: outside, dropped
        (-1.5, 0.0, 0.0),                                   # outside: dropped
        (0.0, 0.0, 0.0),                                    # area = inf below: dropped
    ]
    x = np.concatenate([x, np.array(special, dtype=np.float64).T], axis=1).astype(NP_DT[real])
    area = rng.uniform(0.5, 1.5, size=x.shape[1]).astype(NP_DT[real]) * (2.0 / n) ** 2
    area[-1] = np.inf
    return faces, (True, True, False), x, area, 6, 2


@pytest.mark.parametrize("real", ["f64", "f32"])
@pytest.mark.parametrize("method", ["exact", "fast"])
def test_edge_markers(api, real, method):
    rng = np.random.default_rng(17)
    n = 16
    faces, periodic, x, area, n_drop, n_nonfinite = _edge_markers(n, rng, real)
    grid = oracle.Grid(faces, periodic)
    M = x.shape[1]
    u = rng.normal(size=(3, n, n, n)).astype(NP_DT[real])
    F = rng.normal(size=(3, M)).astype(NP_DT[real])
    ctx = api.Context(faces, periodic, real=real)
    g = run_gpu(ctx, x, area, method, torch.as_tensor(u, device=DEV), F)
    r = run_oracle(grid, x, area, method, u, F)
    st = g["status"]
    assert st["dropped"] == n_drop and st["nonfinite"] == n_nonfinite
    dropped = ~r["tr"].sup.ok
    assert dropped.sum() == n_drop
    assert np.array_equal(g["home"], home_linear(r["tr"].sup, grid.n))
    assert np.all(g["phi"][dropped] == 0) and np.all(g["c"][dropped] == 0) and np.all(g["U"][:, dropped] == 0)
    if method == "fast" and real == "f32":
        fixed = r["phi"].copy()
        resolved, unresolved = fast_tie_fix(grid, x, g["phi"], r["phi"], TOL[real], fixed=fixed)
        assert unresolved == 0
        bad = ~np.isfinite(area.astype(np.float64))
        r = oracle_outputs_with_phi(grid, r["tr"], fixed, np.where(bad, 0.0, area), u, F)
    _compare(g, r, TOL[real])


def test_empty_and_capacity(api):
    faces = [uniform_faces(8)] * 3
    ctx = api.Context(faces, (True, True, True), real="f32")
    T = ctx.transfer(10)
    x = torch.empty((3, 0), dtype=torch.float32, device=DEV)
    a = torch.empty((0,), dtype=torch.float32, device=DEV)
    ctx.build_transfer(T, x, a)
    u = torch.ones((3, 8, 8, 8), dtype=torch.float32, device=DEV)
    assert ctx.interpolate(T, u).shape == (3, 0)
    f = torch.zeros_like(u)
    ctx.spread(T, torch.empty((3, 0), dtype=torch.float32, device=DEV), f)
    assert ctx.status(T)["dropped"] == 0 and float(f.abs().sum()) == 0.0
    from paper_1805_01113_gb300 import binding as B
    x11 = torch.zeros((3, 11), dtype=torch.float32, device=DEV)
    with pytest.raises(B.MlsError) as e:
        ctx.build_transfer(T, x11, torch.ones(11, dtype=torch.float32, device=DEV))
    assert e.value.code == B.MLS_ERR_CAPACITY


def test_crowded_tile(api):
    """3000 markers inside two cells: one tile split over many blocks and runs."""
    rng = np.random.default_rng(5)
    n = 24
    faces = [uniform_faces(n)] * 3
    grid = oracle.Grid(faces, (True, True, True))
    h = 2.0 / n
    x = (-1.0 + h * np.array([[9.0], [9.0], [9.0]]) + rng.uniform(0, [[2 * h], [h], [h]], size=(3, 3000)))
    x = x.astype(np.float32)
    area = np.full(3000, 0.01 * h * h, dtype=np.float32)
    u = rng.normal(size=(3, n, n, n)).astype(np.float32)
    F = rng.normal(size=(3, 3000)).astype(np.float32)
    ctx = api.Context(faces, (True, True, True), real="f32")
    g = run_gpu(ctx, x, area, "exact", torch.as_tensor(u, device=DEV), F)
    r = run_oracle(grid, x, area, "exact", u, F)
    _compare(g, r, TOL["f32"])


@pytest.mark.parametrize("nx", [21, 22])
def test_uneven_x_extent(api, nx):
    """n_x odd (scalar-load interpolation, scalar flush) and n_x = 2 mod 4 (paired loads, scalar flush),
    with markers on both periodic x seams."""
    rng = np.random.default_rng(nx)
    faces = [uniform_faces(nx), uniform_faces(16), uniform_faces(12)]
    periodic = (True, True, True)
    grid = oracle.Grid(faces, periodic)
    M = 4000
    x = np.stack([rng.uniform(-1, 1, M) for _ in range(3)])
    x[0, :200] = rng.uniform(faces[0][0], faces[0][1], 200)         # home cell x = 0
    x[0, 200:400] = rng.uniform(faces[0][nx - 1], faces[0][nx], 200)  # home cell x = n_x - 1
    x = x.astype(np.float32)
    x[0] = np.minimum(x[0], _below(faces[0][nx], "f32"))
    area = rng.uniform(0.5, 1.5, M).astype(np.float32) * (2.0 / 16) ** 2
    u = rng.normal(size=(3, 12, 16, nx)).astype(np.float32)
    F = rng.normal(size=(3, M)).astype(np.float32)
    ctx = api.Context(faces, periodic, real="f32", brick_log2=(2, 2, 2))
    g = run_gpu(ctx, x, area, "exact", torch.as_tensor(u, device=DEV), F)
    r = run_oracle(grid, x, area, "exact", u, F)
    assert g["status"]["dropped"] == 0
    _compare(g, r, TOL["f32"])


@pytest.mark.parametrize("brick", [(1, 1, 1), (2, 3, 4), (5, 5, 1)])
def test_tile_shapes(api, brick):
    w = make_workload("c2", n=64, n_bodies=12)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = field_full_np(w.modes, w.faces, np.float32)
    F = w.forces().astype(np.float32)
    ctx = api.Context(w.faces, w.periodic, real="f32", brick_log2=brick)
    g = run_gpu(ctx, x, area, "exact", torch.as_tensor(u, device=DEV), F)
    r = run_oracle(grid, x, area, "exact", u, F)
    _compare(g, r, TOL["f32"])


def test_double_fallback_on_conditioning(api):
    """cond_max = 1 forces every single-precision solve through the double path."""
    w = make_workload("c2", n=64, n_bodies=6)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    ctx = api.Context(w.faces, w.periodic, real="f32", cond_max=1.0)
    g = run_gpu(ctx, x, area, "exact")
    r = run_oracle(grid, x, area, "exact")
    assert g["status"]["refined_fp64"] == x.shape[1]
    assert normwise(g["phi"], r["phi"]) <= 1e-6
    ctx2 = api.Context(w.faces, w.periodic, real="f32")
    assert run_gpu(ctx2, x, area, "exact")["status"]["refined_fp64"] == 0


def _narrow_cells_grid(r=8.0):
    """Periodic uniform x, y (16 cells); z walled, 16 cells whose widths are r
    except three narrow ones (cells 3, 7, 11, width 1): in a narrow cell the
    neighbours lie (1 + r)/2 home widths away, where the Gaussian is tiny, so
    A is nearly singular in z."""
    w = np.full(16, r)
    w[[3, 7, 11]] = 1.0
    fz = np.concatenate([[0.0], np.cumsum(w)])
    return [uniform_faces(16), uniform_faces(16), fz / fz[-1] * 2 - 1], (True, True, False)


def test_double_resolve_decided_by_data(api):
    """Near-degenerate supports (narrow cells between cells 8 times wider):
    cond_1(A) passes 1e6 by itself for most markers in the narrow cells and
    stays O(1-100) elsewhere.  The single-precision build re-solves in double
    exactly the markers whose condition number exceeds cond_max (counted
    against the oracle's cond_1, with a +/-25 % band for the single-precision
    estimate), and those markers meet the single-precision tolerance.  The
    float path itself (one refinement step in float) holds the tolerance only
    up to cond_1 of about 1e3 (its error grows like cond_1 times the float
    epsilon), so cond_max = 1e3 keeps every marker within it."""
    faces, periodic = _narrow_cells_grid()
    grid = oracle.Grid(faces, periodic)
    rng = np.random.default_rng(77)
    fz = faces[2]
    narrow = [3, 7, 11]
    zc = np.concatenate([rng.uniform(fz[c], fz[c + 1], 400) for c in narrow]
                        + [rng.uniform(fz[c], fz[c + 1], 100) for c in (1, 5, 9, 13, 14)])
    K = zc.shape[0]
    x = np.stack([rng.uniform(-0.9, 0.9, K), rng.uniform(-0.9, 0.9, K), zc]).astype(np.float32)
    area = np.full(K, 1e-3, dtype=np.float32)
    _, cond = oracle.moment_matrix(grid, x.astype(np.float64), 1.0)
    assert np.all(np.isfinite(cond))
    r = run_oracle(grid, x, area, "exact")
    scale = np.max(np.abs(r["phi"]))
    report = []
    for cmax in (1e6, 1e3):
        lo, hi = int((cond > 1.25 * cmax).sum()), int((cond > 0.8 * cmax).sum())
        assert lo > 500 and hi < K
        ctx = api.Context(faces, periodic, real="f32", cond_max=cmax)
        g = run_gpu(ctx, x, area, "exact")
        assert g["status"]["dropped"] == 0
        assert lo <= g["status"]["refined_fp64"] <= hi
        err = np.max(np.abs(g["phi"] - r["phi"]), axis=1) / scale
        assert np.max(err[cond > 1.25 * cmax]) <= TOL["f32"]            # re-solved in double
        assert np.max(err[cond < 1e3]) <= TOL["f32"]                    # well-conditioned, float path
        mid = (cond >= 1e3) & (cond <= 0.8 * cmax)
        report.append(f"cond_max {cmax:.0e}: re-solved {g['status']['refined_fp64']} of {K} (oracle {lo}..{hi}); "
                      f"max phi error {np.max(err):.2e}, float path with 1e3 <= cond <= {0.8 * cmax:.0e}: "
                      f"{np.max(err[mid], initial=0.0):.2e}")
        if cmax == 1e3:
            assert np.max(err) <= TOL["f32"]
    print("; ".join(report))


@pytest.mark.parametrize("brick", [(3, 3, 3), (1, 3, 3)])
def test_bf16_fields(api, brick):
    """bfloat16 field storage with float accumulation: interpolation from identical inputs
    stays at single-precision accuracy; the spread field is rounded to bfloat16 (8-byte
    bf16x2 vector reductions with 8x8x8 tiles, scalar ones with 2-wide tiles)."""
    w = make_workload("c2", n=64, n_bodies=12)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = torch.as_tensor(field_full_np(w.modes, w.faces), device=DEV).to(torch.bfloat16)
    F = w.forces().astype(np.float32)
    ctx = api.Context(w.faces, w.periodic, real="f32", field="bf16", brick_log2=brick)
    g = run_gpu(ctx, x, area, "exact", u, F)
    r = run_oracle(grid, x, area, "exact", u.double().cpu().numpy(), F)
    assert normwise(g["U"], r["U"]) <= TOL["f32"]
    assert normwise(g["f"], r["f"]) <= 1e-2


@pytest.mark.parametrize("layout", ["walled_x", "odd_x"])
def test_bf16_fields_pair_staging_edges(api, layout):
    """The bfloat16 interpolation brick is copied in 4-byte pairs of cells when
    the x extent is even: pairs that would leave a walled x axis are skipped,
    and an odd x extent falls back to cell-by-cell copies.  Interpolation from
    identical bfloat16 inputs stays at single-precision accuracy either way."""
    w = make_workload("c2", n=64, n_bodies=12)
    if layout == "walled_x":
        faces, periodic = w.faces, (False, True, True)
    else:
        faces, periodic = (uniform_faces(63), w.faces[1], w.faces[2]), w.periodic
    grid = oracle.Grid(faces, periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = torch.as_tensor(field_full_np(w.modes, faces), device=DEV).to(torch.bfloat16)
    F = w.forces().astype(np.float32)
    for brick in [(3, 3, 3), (2, 3, 2)]:
        ctx = api.Context(faces, periodic, real="f32", field="bf16", brick_log2=brick)
        g = run_gpu(ctx, x, area, "exact", u, F)
        r = run_oracle(grid, x, area, "exact", u.double().cpu().numpy(), F)
        assert g["status"]["dropped"] == 0
        assert normwise(g["U"], r["U"]) <= TOL["f32"]
        assert normwise(g["f"], r["f"]) <= 1e-2


def test_rebuild_is_deterministic_per_marker(api):
    w = make_workload("c2", n=64, n_bodies=10)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = torch.as_tensor(field_full_np(w.modes, w.faces, np.float32), device=DEV)
    ctx = api.Context(w.faces, w.periodic, real="f32")
    T = ctx.transfer(x.shape[1])
    a = run_gpu(ctx, x, area, "exact", u, T=T)
    b = run_gpu(ctx, x, area, "exact", u, T=T)
    assert np.array_equal(a["phi"], b["phi"]) and np.array_equal(a["U"], b["U"])


def test_rebuild_with_other_markers(api):
    """One transfer rebuilt on marker sets of different sizes and places gives
    what a fresh transfer gives: nothing of a previous build's tile sort (bin
    counts, offsets, tile list) leaks into the next."""
    w = make_workload("c2", n=64, n_bodies=12)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = torch.as_tensor(field_full_np(w.modes, w.faces, np.float32), device=DEV)
    F = w.forces().astype(np.float32)
    ctx = api.Context(w.faces, w.periodic, real="f32")
    T = ctx.transfer(x.shape[1])
    M = x.shape[1]
    for sel in (slice(0, M), slice(M // 3, M // 2), slice(0, 7), slice(M // 4, M)):
        xs, As, Fs = np.ascontiguousarray(x[:, sel]), np.ascontiguousarray(area[sel]), np.ascontiguousarray(F[:, sel])
        got = run_gpu(ctx, xs, As, "exact", u, Fs, T=T)
        ref = run_gpu(ctx, xs, As, "exact", u, Fs)
        assert np.array_equal(got["home"], ref["home"])
        assert normwise(got["phi"], ref["phi"]) <= 1e-6 and normwise(got["U"], ref["U"]) <= 1e-6
        # The spread's fixed-point quantum follows the largest force of each
        # 128-marker chunk, and the order inside a tile (hence the chunks)
        # follows the locate kernel's atomics: rounding differs, a leak would not.
        assert normwise(got["f"], ref["f"]) <= TOL["f32"]


def test_contexts_with_large_tiles_keep_their_shared_memory(api):
    """A kernel's dynamic shared-memory limit is shared by every context: a
    context created later with smaller (but still large) tiles of the same
    kernel must not lower it under an earlier one.  Tiles 4,4,4 need about
    97 KB of spreading accumulator, tiles 4,3,4 about 54 KB."""
    w = make_workload("c2", n=64, n_bodies=6)
    grid = oracle.Grid(w.faces, w.periodic)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    u = field_full_np(w.modes, w.faces, np.float32)
    F = w.forces().astype(np.float32)
    big = api.Context(w.faces, w.periodic, real="f32", brick_log2=(4, 4, 4))
    small = api.Context(w.faces, w.periodic, real="f32", brick_log2=(4, 3, 4))
    r = run_oracle(grid, x, area, "exact", u, F)
    for ctx in (big, small, big):
        g = run_gpu(ctx, x, area, "exact", torch.as_tensor(u, device=DEV), F)
        _compare(g, r, TOL["f32"])


def _neighbour_markers(home3, n, cell):
    """Indices of markers whose home cell lies within +/-1 (periodic) of `cell`."""
    d = [(home3[a] - cell[a] + 1) % n[a] for a in range(3)]
    return np.nonzero((d[0] <= 2) & (d[1] <= 2) & (d[2] <= 2))[0]


def test_full_size_multibody_sampled(api):
    """2000 ellipsoids (2.56 M markers) in 512^3, the benchmark's workload and launch shape."""
    w = make_workload("c2")
    grid = oracle.Grid(w.faces, w.periodic)
    n = grid.n
    M = w.n_markers
    ctx = api.Context(w.faces, w.periodic, real="f32")
    V32 = w.vertices.astype(np.float32)
    x, area = ctx.marker_prep(torch.as_tensor(V32, device=DEV), torch.as_tensor(w.tri, device=DEV))
    u = field_full_torch(w.modes, w.faces, torch.float32, DEV)
    F = torch.as_tensor(w.forces().astype(np.float32), device=DEV)
    T = ctx.transfer(M)
    ctx.build_transfer(T, x, area, "exact")
    U = ctx.interpolate(T, u)
    f = torch.zeros_like(u)
    ctx.spread(T, F, f)
    assert ctx.status(T)["dropped"] == 0
    phi_g, c_g, _ = __import__("gpu_helpers").gpu_transfer(ctx, T)

    rng = np.random.default_rng(99)
    s = rng.choice(M, size=2000, replace=False)
    xs, as_ = oracle.marker_prep(V32, w.tri[s], "f32")
    assert np.array_equal(x[:, s].cpu().numpy(), xs)
    tr = oracle.shape_exact(grid, xs, 1.0)
    cs = oracle.forcing_scale(tr, as_)
    assert normwise(phi_g[s], tr.phi) <= TOL["f32"]
    assert normwise(c_g[s], cs) <= TOL["f32"]
    ix, iy, iz = (torch.as_tensor(a, device=DEV) for a in tr.sup.idx)
    usup = u[:, iz, iy, ix].double().cpu().numpy()               # input bytes at the supports
    U_ref = np.einsum("mk,cmk->cm", tr.phi, usup)
    assert normwise(U[:, s].double().cpu().numpy(), U_ref) <= TOL["f32"]

    # Spread, element by element on sampled touched cells: every marker whose
    # support covers the cell, recomputed by the oracle.
    xall = x.double().cpu().numpy()
    home3, ok = oracle.locate(grid, xall)
    assert ok.all()
    Fh = F.double().cpu().numpy()
    areah = area.double().cpu().numpy()
    fh_nonzero = torch.nonzero(f[0].reshape(-1) != 0).squeeze(1).cpu().numpy()
    cells = rng.choice(fh_nonzero, size=150, replace=False)
    ref, got = [], []
    fflat = f.reshape(3, -1)
    for key in cells:
        cell = (key % n[0], (key // n[0]) % n[1], key // (n[0] * n[1]))
        ml = _neighbour_markers(home3, n, cell)
        trm = oracle.shape_exact(grid, xall[:, ml], 1.0)
        cm = oracle.forcing_scale(trm, areah[ml])
        lin = (trm.sup.idx[2] * n[1] + trm.sup.idx[1]) * n[0] + trm.sup.idx[0]
        w_ = np.where(lin == key, trm.phi, 0.0).sum(1) * cm
        ref.append((w_[None, :] * Fh[:, ml]).sum(1))
        got.append(fflat[:, key].double().cpu().numpy())
    assert normwise(np.array(got), np.array(ref)) <= TOL["f32"]

    # Conservation (Eq. 7) on a uniform grid: sum_k f_k h^3 = sum_l F_l A_l h.
    h = 2.0 / n[0]
    lhs = f.double().sum(dim=(1, 2, 3)).cpu().numpy() * h ** 3
    rhs = (Fh * areah).sum(1) * h
    scale = (np.abs(Fh) * areah).sum(1) * h
    assert np.all(np.abs(lhs - rhs) <= 1e-5 * scale)
    # Adjointness: <U, c F> = <u, f>.
    v = ctx.view(T)
    cF = torch.zeros_like(F, dtype=torch.float64)
    cF[:, v["perm"].long()] = v["c"].double()[None, :] * F.double()[:, v["perm"].long()]
    a1 = float((U.double() * cF).sum())
    a2 = float((u.double() * f.double()).sum())
    a_scale = float((U.double().abs() * cF.abs()).sum())
    assert abs(a1 - a2) <= 1e-5 * a_scale


def _cells_near(order, keys, n, cell, periodic):
    """Indices of markers (sorted home keys `keys`, permutation `order`) whose home
    cell lies within +/-1 of `cell`, wrapping only the periodic axes."""
    out = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                c = [cell[0] + dx, cell[1] + dy, cell[2] + dz]
                ok = True
                for a in range(3):
                    if periodic[a]:
                        c[a] %= n[a]
                    elif not 0 <= c[a] < n[a]:
                        ok = False
                if not ok:
                    continue
                k = (c[2] * n[1] + c[1]) * n[0] + c[0]
                lo, hi = np.searchsorted(keys, k, "left"), np.searchsorted(keys, k, "right")
                out.append(order[lo:hi])
    return np.concatenate(out) if out else np.zeros(0, dtype=np.int64)


def test_full_size_batched_stretched_sampled(api):
    """10^4 deformed bodies (32 M markers) in 1024^3, tanh-stretched and walled in z:
    the benchmark's headline workload in its launch configuration (autotuned tiles).
    Each field has 3 x 2^30 values, so component offsets pass 2^31; sampled
    markers and cells include the top and bottom z-planes that bodies reach."""
    from paper_1805_01113_gb300 import autotune
    w = make_workload("c3")
    grid = oracle.Grid(w.faces, w.periodic)
    n = grid.n
    M = w.n_markers
    V32 = w.vertices.astype(np.float32)
    prep = api.Context(w.faces, w.periodic, real="f32")
    x, area = prep.marker_prep(torch.as_tensor(V32, device=DEV), torch.as_tensor(w.tri, device=DEV))
    u = field_full_torch(w.modes, w.faces, torch.float32, DEV)
    F = torch.as_tensor(w.forces().astype(np.float32), device=DEV)
    tiles, _ = autotune.tune(w.faces, w.periodic, x, area, u, F, "exact", "f32")
    ctx = api.Context(w.faces, w.periodic, real="f32", brick_log2=tiles)
    T = ctx.transfer(M)
    ctx.build_transfer(T, x, area, "exact")
    U = ctx.interpolate(T, u)
    f = torch.zeros_like(u)
    ctx.spread(T, F, f)
    assert ctx.status(T)["dropped"] == 0
    phi_g, c_g, home_g = __import__("gpu_helpers").gpu_transfer(ctx, T)

    xall = x.double().cpu().numpy()
    home3, ok = oracle.locate(grid, xall)
    assert ok.all()
    key = (home3[2].astype(np.int64) * n[1] + home3[1]) * n[0] + home3[0]
    assert np.array_equal(home_g, key)
    # 2000 sampled markers: random ones plus the lowest and highest in z.
    rng = np.random.default_rng(1805)
    zorder = np.argsort(xall[2], kind="stable")
    s = np.unique(np.concatenate([rng.choice(M, size=1800, replace=False), zorder[:100], zorder[-100:]]))
    xs, as_ = oracle.marker_prep(V32, w.tri[s], "f32")
    assert np.array_equal(x[:, s].cpu().numpy(), xs)
    tr = oracle.shape_exact(grid, xs, 1.0)
    cs = oracle.forcing_scale(tr, as_)
    assert normwise(phi_g[s], tr.phi) <= TOL["f32"]
    assert normwise(c_g[s], cs) <= TOL["f32"]
    ix, iy, iz = (torch.as_tensor(a, device=DEV) for a in tr.sup.idx)
    usup = u[:, iz, iy, ix].double().cpu().numpy()
    U_ref = np.einsum("mk,cmk->cm", tr.phi, usup)
    assert normwise(U[:, s].double().cpu().numpy(), U_ref) <= TOL["f32"]

    # Spread on sampled touched cells (random ones, plus the top and bottom
    # touched z-planes), recomputed by the oracle from every marker whose
    # support covers the cell.
    order = np.argsort(key, kind="stable")
    keys = key[order]
    Fh = F.double().cpu().numpy()
    areah = area.double().cpu().numpy()
    touched_z = torch.nonzero(f[0].reshape(n[2], -1).ne(0).any(dim=1)).squeeze(1).cpu().numpy()
    fflat = f.reshape(3, -1)
    plane = n[0] * n[1]
    cand = [rng.choice(torch.nonzero(f[0].reshape(-1) != 0).squeeze(1).cpu().numpy(), size=130, replace=False)]
    for zp in (touched_z.min(), touched_z.max()):
        nz_in = torch.nonzero(fflat[0, zp * plane:(zp + 1) * plane] != 0).squeeze(1).cpu().numpy() + zp * plane
        cand.append(rng.choice(nz_in, size=min(10, len(nz_in)), replace=False))
    cells = np.concatenate(cand)
    ref, got = [], []
    for kc in cells:
        cell = (int(kc % n[0]), int((kc // n[0]) % n[1]), int(kc // plane))
        ml = _cells_near(order, keys, n, cell, w.periodic)
        trm = oracle.shape_exact(grid, xall[:, ml], 1.0)
        cm = oracle.forcing_scale(trm, areah[ml])
        lin = (trm.sup.idx[2] * n[1] + trm.sup.idx[1]) * n[0] + trm.sup.idx[0]
        w_ = np.where(lin == kc, trm.phi, 0.0).sum(1) * cm
        ref.append((w_[None, :] * Fh[:, ml]).sum(1))
        got.append(fflat[:, kc].double().cpu().numpy())
    assert normwise(np.array(got), np.array(ref)) <= TOL["f32"]

    # Conservation (Eq. 7) with the GPU's phi and c: sum_k f_k dV_k equals
    # sum_l c_l F_l sum_k phi_k^l dV_k (= sum_l F_l dV_l), on a stretched grid.
    wz = torch.as_tensor(grid.widths[2], device=DEV)
    hxy = float(grid.widths[0][0] * grid.widths[1][0])
    lhs = np.array([float((f[q].double().sum(dim=(1, 2)) * wz).sum()) for q in range(3)]) * hxy
    v = ctx.view(T)
    hz = (v["home"].long() // plane)
    dvk = torch.stack([wz[(hz + dz).clamp(0, n[2] - 1)] for dz in (-1, 0, 1)])  # (3, M)
    ph = v["phi"].double().reshape(3, 9, -1).sum(1)                              # sum over the 9 x,y nodes per z
    sdv = (ph * dvk).sum(0) * hxy
    cF = v["c"].double()[None, :] * F.double()[:, v["perm"].long()]
    rhs = (cF * sdv[None, :]).sum(1).cpu().numpy()
    scale = (cF.abs() * sdv[None, :].abs()).sum(1).cpu().numpy()
    assert np.all(np.abs(lhs - rhs) <= 1e-5 * scale)
    # Adjointness: <U, c F> = <u, f>.
    cFc = torch.zeros_like(F, dtype=torch.float64)
    cFc[:, v["perm"].long()] = cF
    a1 = float((U.double() * cFc).sum())
    a2 = sum(float((u[q].double() * f[q].double()).sum()) for q in range(3))
    a_scale = float((U.double().abs() * cFc.abs()).sum())
    assert abs(a1 - a2) <= 1e-5 * a_scale
