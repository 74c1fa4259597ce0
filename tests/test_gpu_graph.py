"""The batched step captured once in a CUDA graph and replayed on new data.

A solver captures its time step (marker prep from the triangle vertices,
exact-MLS build, interpolation, spreading) once and replays it every step
after copying the new vertex positions and marker forces into the captured
buffers.  This checks that each replay recomputes everything from the buffers'
current contents: after two replays on moved bodies and new forces, the
marker velocities and the spread field match the CPU oracle on those inputs.
"""

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import DEV, normwise
from workloads import make_workload
from workloads.fields import field_full_np

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_01113_gb300 import api as _api
    torch.cuda.set_device(0)
    return _api


@pytest.mark.parametrize("calls", ["separate", "build_interpolate", "build_direct_forcing"])
def test_graph_replay_on_new_positions_and_forces(api, calls):
    """The step through the three calls, through mls_build_interpolate (the
    benchmark's headline), and the direct-forcing step through
    mls_build_direct_forcing (forces F = (V_b - U)/dt)."""
    w = make_workload("c3", n=96, n_bodies=16)
    grid = oracle.Grid(w.faces, w.periodic)
    M = w.n_markers
    V0 = w.vertices.astype(np.float32)
    u_np = field_full_np(w.modes, w.faces, np.float32)
    ctx = api.Context(w.faces, w.periodic, real="f32", brick_log2=(3, 3, 2))
    V = torch.as_tensor(V0, device=DEV)
    tri = torch.as_tensor(w.tri, device=DEV)
    F = torch.as_tensor(w.forces().astype(np.float32), device=DEV)
    u = torch.as_tensor(u_np, device=DEV)
    x = torch.empty((3, M), dtype=torch.float32, device=DEV)
    area = torch.empty((M,), dtype=torch.float32, device=DEV)
    U = torch.empty((3, M), dtype=torch.float32, device=DEV)
    f = torch.zeros_like(u)
    T = ctx.transfer(M)

    Vb = torch.zeros((3, M), dtype=torch.float32, device=DEV)
    Fo = torch.empty((3, M), dtype=torch.float32, device=DEV)
    dt = 0.5

    def step():
        f.zero_()
        ctx.marker_prep(V, tri, x, area)
        if calls == "separate":
            ctx.build_transfer(T, x, area, "exact")
            ctx.interpolate(T, u, U)
            ctx.spread(T, F, f)
        elif calls == "build_interpolate":
            ctx.build_interpolate(T, x, area, u, U, method="exact")
            ctx.spread(T, F, f)
        else:
            ctx.build_direct_forcing(T, x, area, u, Vb, dt, f, F=Fo, U=U, method="exact")

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()                                        # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()

    rng = np.random.default_rng(2024)
    h = 2.0 / 96
    for rep in range(2):
        # Move every body by its own sub-cell shift (z kept inside the walls) and draw new forces.
        shift = rng.uniform(-0.7 * h, 0.7 * h, size=(len(w.body_faces) - 1, 3))
        shift[:, 2] *= 0.5
        Vn = V0.astype(np.float64).copy()
        # vertex ranges per body: faces of body b reference its own vertices only
        for b in range(len(w.body_faces) - 1):
            t0, t1 = int(w.body_faces[b]), int(w.body_faces[b + 1])
            vids = np.unique(w.tri[t0:t1])
            Vn[vids] += shift[b]
        Vn = Vn.astype(np.float32)
        Fn = rng.normal(size=(3, M)).astype(np.float32)
        Vbn = rng.normal(size=(3, M)).astype(np.float32)
        V.copy_(torch.as_tensor(Vn))
        F.copy_(torch.as_tensor(Fn))
        Vb.copy_(torch.as_tensor(Vbn))
        g.replay()
        torch.cuda.synchronize()
        assert ctx.status(T)["dropped"] == 0
        xr, ar = oracle.marker_prep(Vn, w.tri, "f32")
        assert np.array_equal(x.cpu().numpy(), xr)
        tr = oracle.shape_exact(grid, xr, 1.0)
        c = oracle.forcing_scale(tr, ar)
        U_ref = oracle.interpolate(tr, u_np.astype(np.float64))
        if calls == "build_direct_forcing":
            U_ref, F_ref, sp = oracle.direct_forcing(tr, c, u_np.astype(np.float64), Vbn.astype(np.float64), dt,
                                                     grid.n)
            f_ref = sp.to_dense(grid.n)
            assert normwise(Fo.double().cpu().numpy(), F_ref) <= TOL
        else:
            f_ref = oracle.spread(tr, c, Fn.astype(np.float64), grid.n).to_dense(grid.n)
        assert normwise(U.double().cpu().numpy(), U_ref) <= TOL
        fg = f.double().cpu().numpy()
        assert normwise(fg, f_ref) <= TOL
        assert np.all(fg[f_ref == 0] == 0)             # untouched cells stay exactly zero
