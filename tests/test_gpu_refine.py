"""Adaptive Lagrangian refinement (mls_refine_markers) against the CPU oracle.

Levels and parents are integers decided in double precision from the
working-precision areas on both sides: bit-exact.  Refined centroids and areas
use the same operation order as the oracle's marker definition: bit-exact in
float32 and float64.
"""

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import DEV, NP_DT, TORCH_DT
from oracle.refine import refine, refine_levels
from workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_01113_gb300 import api as _api
    torch.cuda.set_device(0)
    return _api


@pytest.mark.parametrize("real", ["f32", "f64"])
@pytest.mark.parametrize("ratio,max_level", [(0.8, 3), (1.5, 3), (0.4, 3), (0.8, 1)])
def test_refine_matches_oracle(api, real, ratio, max_level):
    w = make_workload("c3", n=64, n_bodies=8)                # mixed icosphere levels, stretched z
    grid = oracle.Grid(w.faces, w.periodic)
    V = w.vertices.astype(NP_DT[real])
    ctx = api.Context(w.faces, w.periodic, real=real)
    x, area, parent, level = ctx.refine_markers(torch.as_tensor(V, device=DEV), torch.as_tensor(w.tri, device=DEV),
                                                ratio=ratio, max_level=max_level)
    torch.cuda.synchronize()
    lev_r = refine_levels(grid, V, w.tri, ratio=ratio, max_level=max_level, precision=real)
    assert np.array_equal(level.cpu().numpy(), lev_r)
    xr, ar, pr = refine(V, w.tri, lev_r, precision=real)
    assert np.array_equal(parent.cpu().numpy(), pr)
    assert np.array_equal(x.cpu().numpy(), xr)
    assert np.array_equal(area.cpu().numpy(), ar)
    if max_level == 3 and ratio == 0.8:
        assert len(np.unique(lev_r)) >= 2                   # a mix of levels


def test_capacity_and_build(api):
    from paper_1805_01113_gb300 import binding as B
    w = make_workload("c2", n=64, n_bodies=4)
    ctx = api.Context(w.faces, w.periodic, real="f32")
    V = torch.as_tensor(w.vertices.astype(np.float32), device=DEV)
    tri = torch.as_tensor(w.tri, device=DEV)
    with pytest.raises(B.MlsError) as e:
        ctx.refine_markers(V, tri, ratio=0.5, capacity=w.tri.shape[0])
    assert e.value.code == B.MLS_ERR_CAPACITY
    x, area, parent, level = ctx.refine_markers(V, tri, ratio=0.5)
    assert x.shape[1] == int((level + 1).sum().item())
    # The refined markers feed the build: the forcing volume of each base
    # triangle is shared by its pieces (sum of refined areas = base area).
    T = ctx.transfer(x.shape[1])
    ctx.build_transfer(T, x, area)
    assert ctx.status(T)["dropped"] == 0
    xb, ab = ctx.marker_prep(V, tri)
    sums = torch.zeros_like(ab).index_add_(0, parent.long(), area)
    assert float(((sums - ab).abs() / ab).max()) < 1e-5
