"""mls_marker_prep_locate: markers formed from their triangles and located,
piece by piece, ahead of the build that then skips its own locate pass.

The markers equal mls_marker_prep's bit for bit; the build that follows
leaves, marker by marker, the same transfer (phi, c, home) and U as
mls_marker_prep followed by the plain build, with the same counters; the
spread agrees to the fixed-point rounding of its chunks (whose makeup follows
the order the locate atomics give inside a tile).  Pieces out of order are
refused, and a build on other arrays locates its markers itself.
"""

import numpy as np
import pytest
import torch

from gpu_helpers import DEV, NP_DT, gpu_transfer, normwise
from workloads import make_workload
from workloads.fields import field_full_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_01113_gb300 import api as _api
    torch.cuda.set_device(0)
    return _api


def _inputs(w, real, broken=True):
    V = w.vertices.astype(NP_DT[real])
    tri = w.tri.copy()
    if broken:
        tri[5] = [0, 1, len(V)]            # a vertex index out of range: NaN marker (dropped, non-finite)
        V[tri[200, 0]] *= 50.0             # triangles around one vertex: centroids off the grid (dropped)
    return torch.as_tensor(V, device=DEV), torch.as_tensor(tri, device=DEV)


def _pieces(w, cuts):
    bf = np.asarray(w.body_faces)
    t = [int(bf[min(b, len(bf) - 1)]) for b in cuts]
    return list(zip(t[:-1], t[1:]))


def _step(ctx, T, x, area, u, F):
    U = ctx.build_interpolate(T, x, area, u)
    f = torch.zeros_like(u)
    ctx.spread(T, F, f)
    torch.cuda.synchronize()
    out = {"status": ctx.status(T), "U": U.double().cpu().numpy(), "f": f.double().cpu().numpy()}
    out["phi"], out["c"], out["home"] = gpu_transfer(ctx, T)
    return out


def _same_transfer(a, b, f_tol):
    assert a["status"] == b["status"]
    assert np.array_equal(a["home"], b["home"])
    assert np.array_equal(a["phi"], b["phi"]) and np.array_equal(a["c"], b["c"])
    assert np.array_equal(a["U"], b["U"])
    assert normwise(a["f"], b["f"]) <= f_tol


@pytest.mark.parametrize("real", ["f32", "f64"])
def test_pieces_match_prep_then_build(api, real):
    w = (make_workload("c3", n=96, n_bodies=16) if real == "f32"
         else make_workload("c1", n=48, level=3, radius=0.3))
    V, tri = _inputs(w, real)
    nt = tri.shape[0]
    ctx = api.Context(w.faces, w.periodic, real=real)
    dt = ctx.real_t
    u = torch.as_tensor(field_full_np(w.modes, w.faces, NP_DT[real]), device=DEV)
    F = torch.as_tensor(w.forces().astype(NP_DT[real]), device=DEV)

    x, area = ctx.marker_prep(V, tri)
    Ta = ctx.transfer(nt)
    ref = _step(ctx, Ta, x, area, u, F)
    assert ref["status"]["dropped"] > 1 and ref["status"]["nonfinite"] == 1

    xb = torch.full((3, nt), 3.0, dtype=dt, device=DEV)
    ab = torch.full((nt,), 3.0, dtype=dt, device=DEV)
    Tb = ctx.transfer(nt)
    nb = len(w.body_faces) - 1
    cuts = [0, nb // 3, nb // 3 + 1, nb] if nb > 2 else [0, nb]
    ctx.timing(True)
    ctx.read_timing()
    for t0, t1 in _pieces(w, cuts):
        ctx.marker_prep_locate(Tb, V, tri, xb, ab, begin=t0, end=t1)
    got = _step(ctx, Tb, xb, ab, u, F)
    kt = ctx.read_timing()
    ctx.timing(False)
    assert np.array_equal(xb.cpu().numpy(), x.cpu().numpy(), equal_nan=True)
    assert np.array_equal(ab.cpu().numpy(), area.cpu().numpy(), equal_nan=True)
    assert kt.get("locate", (0, 0.0))[0] == 0 and kt["prep_locate"][0] == len(cuts) - 1
    _same_transfer(got, ref, 1e-12 if real == "f64" else 1e-5)
    Ta.close()
    Tb.close()


def test_other_arrays_and_later_builds_locate_themselves(api):
    w = make_workload("c3", n=96, n_bodies=16)
    V, tri = _inputs(w, "f32", broken=False)
    nt = tri.shape[0]
    ctx = api.Context(w.faces, w.periodic, real="f32")
    u = torch.as_tensor(field_full_np(w.modes, w.faces, np.float32), device=DEV)
    F = torch.as_tensor(w.forces().astype(np.float32), device=DEV)
    x, area = ctx.marker_prep(V, tri)
    Ta = ctx.transfer(nt)
    ref = _step(ctx, Ta, x, area, u, F)

    xb, ab = torch.empty_like(x), torch.empty_like(area)
    Tb = ctx.transfer(nt)
    ctx.timing(True)
    ctx.read_timing()
    ctx.marker_prep_locate(Tb, V, tri, xb, ab)
    got = _step(ctx, Tb, x, area, u, F)              # other arrays (same values): the build locates again
    assert ctx.read_timing()["locate"][0] == 1
    _same_transfer(got, ref, 1e-5)
    ctx.marker_prep_locate(Tb, V, tri, xb, ab)
    _step(ctx, Tb, xb, ab, u, F)                     # consumed by this build ...
    assert ctx.read_timing().get("locate", (0, 0.0))[0] == 0
    got = _step(ctx, Tb, xb, ab, u, F)               # ... so the next one locates its markers itself
    assert ctx.read_timing()["locate"][0] == 1
    ctx.timing(False)
    _same_transfer(got, ref, 1e-5)
    Ta.close()
    Tb.close()


def test_pieces_out_of_order_are_refused(api):
    from paper_1805_01113_gb300 import binding as B
    w = make_workload("c2", n=64, n_bodies=10)
    V, tri = _inputs(w, "f32", broken=False)
    nt = tri.shape[0]
    ctx = api.Context(w.faces, w.periodic, real="f32")
    x = torch.empty((3, nt), dtype=torch.float32, device=DEV)
    a = torch.empty((nt,), dtype=torch.float32, device=DEV)
    T = ctx.transfer(nt)
    h = nt // 2

    def refused(code, *args, **kw):
        with pytest.raises(B.MlsError) as e:
            ctx.marker_prep_locate(*args, **kw)
        assert e.value.code == code

    refused(B.MLS_ERR_INVALID_ARG, T, V, tri, x, a, begin=h, end=nt)       # does not start at 0
    ctx.marker_prep_locate(T, V, tri, x, a, begin=0, end=h)
    refused(B.MLS_ERR_INVALID_ARG, T, V, tri, x, a, begin=h + 1, end=nt)   # a gap
    refused(B.MLS_ERR_INVALID_ARG, T, V, tri, torch.empty_like(x), a, begin=h, end=nt)   # other x
    refused(B.MLS_ERR_INVALID_ARG, T, V, tri, x, a, begin=h, end=nt + 1)   # past n_tri
    ctx.marker_prep_locate(T, V, tri, x, a, begin=h, end=nt)               # the right piece still goes
    small = ctx.transfer(nt - 1)
    refused(B.MLS_ERR_CAPACITY, small, V, tri, x, a)
    small.close()
    T.close()


def test_full_size_pieces_four_markers_per_thread(api):
    """2.56 M markers (the locate kernel's four-markers-per-thread form), eight
    pieces of whole bodies: U and the transfer per marker against the plain path."""
    w = make_workload("c2")
    V, tri = _inputs(w, "f32", broken=False)
    nt = tri.shape[0]
    ctx = api.Context(w.faces, w.periodic, real="f32")
    u = torch.as_tensor(field_full_np(w.modes, w.faces, np.float32), device=DEV)
    x, area = ctx.marker_prep(V, tri)
    T = ctx.transfer(nt)
    Ua = ctx.build_interpolate(T, x, area, u).cpu().numpy()
    pa, ca, ha = gpu_transfer(ctx, T)
    xb, ab = torch.empty_like(x), torch.empty_like(area)
    nb = len(w.body_faces) - 1
    for t0, t1 in _pieces(w, [q * nb // 8 for q in range(9)]):
        ctx.marker_prep_locate(T, V, tri, xb, ab, begin=t0, end=t1)
    Ub = ctx.build_interpolate(T, xb, ab, u).cpu().numpy()
    pb, cb, hb = gpu_transfer(ctx, T)
    assert ctx.status(T)["dropped"] == 0
    assert torch.equal(xb, x) and torch.equal(ab, area)
    assert np.array_equal(Ua, Ub) and np.array_equal(ha, hb)
    assert np.array_equal(pa, pb) and np.array_equal(ca, cb)
    T.close()
