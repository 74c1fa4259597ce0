"""The allocation-free build entry point agrees with the regular build.

Some callers cannot call cudaMalloc when they build transfer functions: a
flow solver that hands out all device memory from its own pool, or a time
step in which a device allocation would synchronise the whole GPU.  For them
mls_build_transfer_noalloc writes into buffers the caller already owns and
keeps its sorting workspace in a static device array.  This file calls it
through the C ABI twice in a row, on different marker sets, and compares
each result with mls_build_transfer on the same markers.  It is named so
that pytest collects it last.
"""

import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from workloads import make_workload

pytestmark = pytest.mark.gpu

TOL = 1e-5            # single-precision tolerance of the parity tests
DEV = torch.device("cuda", 0)


def _caller_order(phi, c, home, perm):
    p = perm.cpu().numpy().astype(np.int64)
    M = p.shape[0]
    assert np.array_equal(np.sort(p), np.arange(M))
    out_phi = np.empty((M, 27))
    out_phi[p] = phi.double().cpu().numpy().T
    out_c = np.empty(M)
    out_c[p] = c.double().cpu().numpy()
    out_home = np.empty(M, dtype=np.int64)
    out_home[p] = home.cpu().numpy()
    return out_phi, out_c, out_home


def _normwise(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _noalloc(ctx, x, area, method):
    from paper_1805_01113_gb300 import binding as B
    M = x.shape[1]
    ld = M + 37                                            # a padded leading dimension
    phi = torch.full((27, ld), np.nan, dtype=torch.float32, device=DEV)
    c = torch.full((ld,), np.nan, dtype=torch.float32, device=DEV)
    home = torch.full((ld,), -7, dtype=torch.int32, device=DEV)
    perm = torch.full((ld,), -7, dtype=torch.int32, device=DEV)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = ctx.lib.mls_build_transfer_noalloc(ctx.handle, C.c_void_p(x.data_ptr()), C.c_void_p(area.data_ptr()), M,
                                            {"exact": B.MLS_EXACT, "fast": B.MLS_FAST, "surrogate": B.MLS_SURROGATE}[method],
                                            C.c_void_p(phi.data_ptr()), C.c_void_p(c.data_ptr()),
                                            C.c_void_p(home.data_ptr()), C.c_void_p(perm.data_ptr()), ld, stream)
    B.check(rc, "mls_build_transfer_noalloc")
    torch.cuda.synchronize()
    return _caller_order(phi[:, :M], c[:M], home[:M], perm[:M])


def _regular(ctx, x, area, method):
    T = ctx.transfer(x.shape[1])
    ctx.build_transfer(T, x, area, method)
    v = ctx.view(T)
    out = _caller_order(v["phi"], v["c"], v["home"], v["perm"])
    T.close()
    return out


def test_noalloc_build_matches_regular_build():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_01113_gb300 import api, binding as B
    torch.cuda.set_device(0)
    w = make_workload("c2", n=128, n_bodies=40)          # 51200 markers, 4097 tile bins
    xs, areas = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    ctx = api.Context(w.faces, w.periodic, real="f32")
    # Two calls in a row on different marker sets: the second must not see the
    # first call's leftovers in the shared workspace.
    for sel in (slice(0, 30000), slice(9000, 51200)):
        x = torch.as_tensor(np.ascontiguousarray(xs[:, sel]), device=DEV)
        a = torch.as_tensor(np.ascontiguousarray(areas[sel]), device=DEV)
        got = _noalloc(ctx, x, a, "exact")
        ref = _regular(ctx, x, a, "exact")
        assert np.array_equal(got[2], ref[2])
        assert _normwise(got[0], ref[0]) <= TOL and _normwise(got[1], ref[1]) <= TOL
    # fast-MLS once its table exists (building the table allocates).
    x = torch.as_tensor(np.ascontiguousarray(xs[:, :20000]), device=DEV)
    a = torch.as_tensor(np.ascontiguousarray(areas[:20000]), device=DEV)
    with pytest.raises(B.MlsError) as e:
        _noalloc(ctx, x, a, "fast")
    assert e.value.code == B.MLS_ERR_UNSUPPORTED
    ctx.fast_table()
    got, ref = _noalloc(ctx, x, a, "fast"), _regular(ctx, x, a, "fast")
    assert np.array_equal(got[2], ref[2]) and _normwise(got[0], ref[0]) <= TOL
    # The surrogate is not offered without allocation.
    with pytest.raises(B.MlsError) as e:
        _noalloc(ctx, x, a, "surrogate")
    assert e.value.code == B.MLS_ERR_UNSUPPORTED
    # Sizes beyond the static workspace are refused before any launch.
    big = torch.zeros((3, B.MLS_NOALLOC_MAX_MARKERS + 1), dtype=torch.float32, device=DEV)
    with pytest.raises(B.MlsError) as e:
        _noalloc(ctx, big, torch.ones(big.shape[1], dtype=torch.float32, device=DEV), "exact")
    assert e.value.code == B.MLS_ERR_CAPACITY
