"""Coarse collision detection (mls_collisions) against the CPU oracle, bit-exact.

Cell states and marker flags are integers decided from home cells, which the
single-precision build and the oracle take from the same float32 positions.
"""

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import DEV
from oracle.collision import collision_cells, collision_flags
from workloads import make_workload, uniform_faces

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_01113_gb300 import api as _api
    torch.cuda.set_device(0)
    return _api


def _overlapping_bodies(seed):
    """12 ellipsoids plus shifted copies of two of them (bodies 13, 14), some
    markers without a body (index 0)."""
    rng = np.random.default_rng(seed)
    w = make_workload("c2", n=64, n_bodies=12)
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    bf = np.asarray(w.body_faces)
    body = np.zeros(x.shape[1], dtype=np.int32)
    for b in range(12):
        body[bf[b]:bf[b + 1]] = b + 1
    h = 2.0 / 64
    extra, ebody = [], []
    for k, b in enumerate((0, 5)):
        xs = x[:, bf[b]:bf[b + 1]] + (rng.uniform(-0.6, 0.6, size=(3, 1)) * h).astype(np.float32)
        extra.append(xs)
        ebody.append(np.full(xs.shape[1], 13 + k, dtype=np.int32))
    x = np.concatenate([x] + extra, axis=1).astype(np.float32)
    area = np.concatenate([area] + [area[:e.shape[1]] for e in extra]).astype(np.float32)
    body = np.concatenate([body] + ebody)
    body[rng.choice(body.size, 50, replace=False)] = 0
    return w, x, area, body


@pytest.mark.parametrize("brick", [(3, 3, 3), (3, 3, 2), (1, 2, 3)])
def test_collisions_match_oracle(api, brick):
    w, x, area, body = _overlapping_bodies(1)
    grid = oracle.Grid(w.faces, w.periodic)
    ctx = api.Context(w.faces, w.periodic, real="f32", brick_log2=brick)
    M = x.shape[1]
    T = ctx.transfer(M)
    ctx.build_transfer(T, torch.as_tensor(x, device=DEV), torch.as_tensor(area, device=DEV))
    coll = torch.zeros((64, 64, 64), dtype=torch.int32, device=DEV)
    count = torch.zeros(1, dtype=torch.int64, device=DEV)
    flag = ctx.collisions(T, torch.as_tensor(body, device=DEV), coll=coll, count=count)
    torch.cuda.synchronize()
    home, ok = oracle.locate(grid, x.astype(np.float64))
    want_flags = collision_flags(home, ok, body, grid.n)
    keys, state = collision_cells(home, ok, body, grid.n)
    got = flag.cpu().numpy()
    assert want_flags.sum() > 1000                       # the shifted copies do collide
    assert np.array_equal(got, want_flags)
    assert int(count.item()) == int(want_flags.sum())
    cg = coll.cpu().numpy().ravel()
    assert np.array_equal(np.nonzero(cg)[0], keys)
    assert np.array_equal(cg[keys], state)


def test_no_collisions_and_dropped_markers(api):
    """Separated bodies give no flags; markers outside the grid are never flagged."""
    faces = [uniform_faces(16)] * 3
    grid = oracle.Grid(faces, (True, True, False))
    rng = np.random.default_rng(2)
    x = rng.uniform(-0.9, 0.9, size=(3, 500)).astype(np.float32)
    x[2, :20] = -0.99                                    # wall cell z = 0: no support
    body = np.ones(500, dtype=np.int32)                  # one body
    area = np.full(500, 1e-3, dtype=np.float32)
    ctx = api.Context(faces, (True, True, False), real="f32")
    T = ctx.transfer(500)
    ctx.build_transfer(T, torch.as_tensor(x, device=DEV), torch.as_tensor(area, device=DEV))
    flag = ctx.collisions(T, torch.as_tensor(body, device=DEV))
    assert int(flag.sum().item()) == 0
    home, ok = oracle.locate(grid, x.astype(np.float64))
    assert not ok[:20].any()
    # Two bodies in alternate halves of each cell's population: flags where they share cells.
    body2 = (1 + (np.arange(500) % 2)).astype(np.int32)
    flag2 = ctx.collisions(T, torch.as_tensor(body2, device=DEV)).cpu().numpy()
    assert np.array_equal(flag2, collision_flags(home, ok, body2, grid.n))
    assert not flag2[:20].any()
