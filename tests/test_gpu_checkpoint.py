"""Checkpoint and resume (mls_save / mls_load) through the C ABI.

A context saved after it has built its fast-MLS table (Section 2, Fig. 1b/1c)
and been given surrogate parameters is loaded into a fresh context on the same
grid.  The table and the parameters come back byte for byte.  Fast-MLS and
surrogate builds on the loaded context reproduce the saved context's shape
functions bit for bit, and the loaded context never builds a table of its own.
Files written for another grid or option set, and corrupted or truncated
files, are refused and leave the context unchanged.
"""

import numpy as np
import pytest
import torch

from gpu_helpers import DEV, gpu_transfer
from oracle import mlp
from workloads import tanh_faces, uniform_faces

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_01113_gb300 import api as _api
    torch.cuda.set_device(0)
    return _api


def _grid():
    return ([uniform_faces(40), uniform_faces(32), tanh_faces(48, 1.5)], (True, True, False))


def _markers(faces, M, seed):
    """Markers anywhere in x and y, and far enough from the z walls for their supports to stay inside."""
    rng = np.random.default_rng(seed)
    lo = [faces[0][0], faces[1][0], faces[2][3]]
    hi = [faces[0][-1], faces[1][-1], faces[2][-4]]
    x = np.stack([rng.uniform(lo[d], hi[d], M) for d in range(3)]).astype(np.float32)
    area = rng.uniform(1e-4, 2e-3, M).astype(np.float32)
    return torch.as_tensor(x, device=DEV), torch.as_tensor(area, device=DEV)


def _build(ctx, x, area, method):
    T = ctx.transfer(x.shape[1])
    ctx.build_transfer(T, x, area, method)
    torch.cuda.synchronize()
    phi, c, home = gpu_transfer(ctx, T)
    T.close()
    return phi, c, home


def _theta():
    return (mlp.init_params(7) + 0.02 * np.random.default_rng(3).normal(size=mlp.N_PARAMS)).astype(np.float32)


def test_round_trip_table_and_surrogate(api, tmp_path):
    faces, periodic = _grid()
    x, area = _markers(faces, 5000, 11)
    a = api.Context(faces, periodic, real="f32")
    phi_fast, c_fast, home_fast = _build(a, x, area, "fast")
    a.surrogate_params(_theta())
    phi_sur, c_sur, _ = _build(a, x, area, "surrogate")
    path = tmp_path / "state.mlsckpt"
    a.save(path)
    assert not (tmp_path / "state.mlsckpt.partial").exists()

    b = api.Context(faces, periodic, real="f32")
    b.load(path)
    b.timing(True)
    got_fast, got_c, got_home = _build(b, x, area, "fast")
    assert "fast_table" not in b.read_timing()
    assert np.array_equal(got_fast, phi_fast) and np.array_equal(got_c, c_fast)
    assert np.array_equal(got_home, home_fast)
    assert torch.equal(b.fast_table().cpu(), a.fast_table().cpu())
    assert np.array_equal(b.surrogate_params(), a.surrogate_params())
    got_sur, got_c, _ = _build(b, x, area, "surrogate")
    assert np.array_equal(got_sur, phi_sur) and np.array_equal(got_c, c_sur)


def test_load_over_existing_state(api, tmp_path):
    """Loading into a context that already holds a table and parameters replaces both."""
    faces, periodic = _grid()
    a = api.Context(faces, periodic, real="f32")
    a.fast_table()
    a.surrogate_params(_theta())
    path = tmp_path / "a.mlsckpt"
    a.save(path)
    b = api.Context(faces, periodic, real="f32")
    b.fast_table()
    b.surrogate_params(mlp.init_params(99).astype(np.float32))
    b.load(path)
    assert torch.equal(b.fast_table().cpu(), a.fast_table().cpu())
    assert np.array_equal(b.surrogate_params(), a.surrogate_params())


def test_header_only_checkpoint(api, tmp_path):
    """A context with neither a table nor parameters writes a file that loads and changes nothing."""
    faces, periodic = _grid()
    a = api.Context(faces, periodic, real="f32")
    path = tmp_path / "empty.mlsckpt"
    a.save(path)
    assert path.stat().st_size == 8 + 4 + 4 + 8 + 8
    b = api.Context(faces, periodic, real="f32")
    b.load(path)
    from paper_1805_01113_gb300 import binding as B
    with pytest.raises(B.MlsError) as e:
        b.surrogate_params()
    assert e.value.code == B.MLS_ERR_UNSUPPORTED


@pytest.mark.parametrize("change", ["eps", "n_sub", "real", "face", "periodic", "basis"])
def test_refuses_other_grid_or_options(api, tmp_path, change):
    faces, periodic = _grid()
    a = api.Context(faces, periodic, real="f32")
    a.fast_table()
    path = tmp_path / "a.mlsckpt"
    a.save(path)
    kw = {"real": "f32"}
    f2 = [np.array(f) for f in faces]
    p2 = periodic
    if change == "eps":
        kw["eps"] = 1.25
    elif change == "n_sub":
        kw["n_sub"] = 7
    elif change == "real":
        kw["real"] = "f64"
    elif change == "basis":
        kw["basis"] = 10
    elif change == "face":
        f2[2][10] = np.nextafter(f2[2][10], np.inf)
    else:
        p2 = (True, False, False)
    b = api.Context(f2, p2, **kw)
    from paper_1805_01113_gb300 import binding as B
    with pytest.raises(B.MlsError) as e:
        b.load(path)
    assert e.value.code == B.MLS_ERR_INVALID_ARG
    assert "another grid" in str(e.value)


@pytest.mark.parametrize("damage", ["flip", "truncate", "append", "magic", "missing"])
def test_refuses_damaged_files(api, tmp_path, damage):
    faces, periodic = _grid()
    a = api.Context(faces, periodic, real="f32")
    a.surrogate_params(_theta())
    good = tmp_path / "a.mlsckpt"
    a.save(good)
    raw = bytearray(good.read_bytes())
    bad = tmp_path / "bad.mlsckpt"
    if damage == "flip":
        raw[len(raw) // 2] ^= 0x10
    elif damage == "truncate":
        raw = raw[:-13]
    elif damage == "append":
        raw += b"\0" * 8
    elif damage == "magic":
        raw[0] ^= 0xFF
    if damage != "missing":
        bad.write_bytes(bytes(raw))
    b = api.Context(faces, periodic, real="f32")
    theta_b = mlp.init_params(5).astype(np.float32)
    b.surrogate_params(theta_b)
    from paper_1805_01113_gb300 import binding as B
    with pytest.raises(B.MlsError) as e:
        b.load(bad)
    assert e.value.code == B.MLS_ERR_INVALID_ARG
    assert np.array_equal(b.surrogate_params(), theta_b)
