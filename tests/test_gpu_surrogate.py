"""Learned surrogate on the GPU against the double-precision oracle.

Training points and labels, the float32 loss/gradient (backpropagation) and
forward pass are compared with oracle/mlp.py element by element; the
bfloat16 tensor-core forward within the stated bound; a trained network's
shape functions with exact-MLS and with fast-MLS (n = 9) on the same markers.
"""

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import DEV, gpu_transfer, normwise, run_gpu
from oracle import mlp
from workloads import make_workload, tanh_faces, uniform_faces

pytestmark = pytest.mark.gpu

# bfloat16 keeps 8 significant bits (rounding 2^-9 = 2e-3 relative) on the
# inputs, the weights and the two hidden activations; each layer sums 64 such
# products in float32, so its output carries about sqrt(64) x 2e-3 = 1.6e-2 of
# the typical |w h| terms, and the hidden layers' tanh (hardware approximation,
# about 2^-11 relative) adds less.  Normwise against the largest output, the
# measured difference from the double-precision network is 1.8e-2 to 2.1e-2
# for the trained network's projected phi (test_trained_surrogate_builds
# prints it) and 4.3e-3 for the initial network's forward pass; the bound
# leaves a factor of 1.4 over the largest measurement.
BF16_FORWARD_TOL = 3e-2


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1805_01113_gb300 import api as _api
    torch.cuda.set_device(0)
    return _api


def _grid():
    return ([uniform_faces(48), uniform_faces(48), tanh_faces(48, 1.5)], (True, True, False))


def test_training_samples_match_oracle(api):
    faces, periodic = _grid()
    ctx = api.Context(faces, periodic, real="f32")
    X, T = ctx.surrogate_samples(1000, 3000, 77)
    Xr, Tr = mlp.training_samples(oracle.Grid(faces, periodic), 1000, 3000, 77)
    Xg, Tg = X.double().cpu().numpy(), T.double().cpu().numpy()
    assert np.array_equal(Xg[:, :3], Xr[:, :3])                 # offsets are float32-exact draws
    assert np.max(np.abs(Xg[:, 3:] - Xr[:, 3:])) < 1e-6
    assert np.max(np.abs(Tg - Tr)) < 1e-6


def _batch(faces, periodic, n, seed):
    X, T = mlp.training_samples(oracle.Grid(faces, periodic), 0, n, seed)
    return X.astype(np.float32), T.astype(np.float32)


def test_loss_and_gradient_match_oracle(api):
    faces, periodic = _grid()
    ctx = api.Context(faces, periodic, real="f32")
    theta = (mlp.init_params(5) + 0.05 * np.random.default_rng(1).normal(size=mlp.N_PARAMS)).astype(np.float32)
    ctx.surrogate_params(theta)
    X, T = _batch(faces, periodic, 512, 9)
    loss, g = ctx.surrogate_loss_grad(torch.as_tensor(X, device=DEV), torch.as_tensor(T, device=DEV))
    Lr, gr = mlp.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - Lr) <= 1e-5 * Lr
    assert normwise(g.double().cpu().numpy(), gr) <= 1e-5
    assert np.array_equal(ctx.surrogate_params(), theta)


def test_forward_f32_and_bf16(api):
    faces, periodic = _grid()
    ctx = api.Context(faces, periodic, real="f32")
    theta = mlp.init_params(11).astype(np.float32)
    ctx.surrogate_params(theta)
    X, _ = _batch(faces, periodic, 1000, 13)
    Yr, _ = mlp.forward(theta.astype(np.float64), X.astype(np.float64))
    Xt = torch.as_tensor(X, device=DEV)
    assert normwise(ctx.surrogate_forward(Xt, "f32").double().cpu().numpy(), Yr) <= 1e-5
    e_bf16 = normwise(ctx.surrogate_forward(Xt, "bf16").double().cpu().numpy(), Yr)
    print(f"bf16 forward vs double: {e_bf16:.3e}")
    assert e_bf16 <= BF16_FORWARD_TOL


def test_initialisation_matches_oracle(api):
    faces, periodic = _grid()
    ctx = api.Context(faces, periodic, real="f32")
    ctx.train_surrogate(n_samples=4096, epochs=1, batch=4096, lr=1e-30, lr_final=1e-30, seed=123)
    got = ctx.surrogate_params().astype(np.float64)
    assert np.max(np.abs(got - mlp.init_params(123).astype(np.float32))) < 1e-6


def test_trained_surrogate_builds(api):
    """Train on a stretched grid.  With the gate open (no fallback) the network's
    projected shape functions beat fast-MLS (n = 9) against exact-MLS; at the
    default threshold (1e-4 on the raw output's residual) every fallback marker
    carries exact-MLS, and the fallback rate is reported."""
    w = make_workload("c3", n=96, n_bodies=12)
    grid = oracle.Grid(w.faces, w.periodic)
    ctx = api.Context(w.faces, w.periodic, real="f32", residual_max=1e30)
    loss = ctx.train_surrogate(seed=5)                         # default schedule: 131072 Adam steps
    assert loss < 1e-6
    theta32 = ctx.surrogate_params()
    x, area = oracle.marker_prep(w.vertices.astype(np.float32), w.tri, "f32")
    sel = np.random.default_rng(3).choice(x.shape[1], size=4000, replace=False)
    xs, as_ = np.ascontiguousarray(x[:, sel]), np.ascontiguousarray(area[sel])
    g = run_gpu(ctx, xs, as_, "surrogate")
    ex = oracle.shape_exact(grid, xs, 1.0).phi
    fa = oracle.shape_fast(grid, xs, 1.0, 9).phi
    err_sur = normwise(g["phi"], ex)
    err_fast = normwise(fa, ex)
    scale = np.max(np.abs(ex))
    rms_sur = np.sqrt(np.mean((g["phi"] - ex) ** 2)) / scale
    rms_fast = np.sqrt(np.mean((fa - ex) ** 2)) / scale
    assert g["status"]["dropped"] == 0 and g["status"]["surrogate_fallback"] == 0
    # The gain over fast-MLS (the paper's cheap form): smaller error, max and RMS.
    assert err_sur < err_fast and rms_sur < rms_fast
    # Linear reproduction holds by construction (projection).
    assert np.max(np.abs(g["phi"].sum(1) - 1.0)) < 1e-5
    # Same network in double precision (oracle forward + projection): the GPU
    # differs by the bfloat16 evaluation only.
    theta = theta32.astype(np.float64)
    tr, fb = mlp.shape_surrogate(grid, xs, theta, residual_max=1e30)
    bf16_err = normwise(g["phi"], tr.phi)
    assert bf16_err <= BF16_FORWARD_TOL
    # Default gate: the raw residual of the trained network's outputs decides.
    cd = api.Context(w.faces, w.periodic, real="f32")
    cd.surrogate_params(theta32)
    gd = run_gpu(cd, xs, as_, "surrogate")
    nfb = gd["status"]["surrogate_fallback"]
    took_exact = np.max(np.abs(gd["phi"] - ex), axis=1) <= 1e-5 * scale
    assert took_exact.sum() >= nfb                               # every fallback marker is exact-MLS
    _, fbr = mlp.shape_surrogate(grid, xs, theta)                 # oracle's decision (double precision)
    print(f"surrogate error {err_sur:.3e} (rms {rms_sur:.3e}), fast-MLS error {err_fast:.3e} "
          f"(rms {rms_fast:.3e}), loss {loss:.3e}, bf16 vs double {bf16_err:.3e}; default gate: fallback "
          f"{nfb}/{xs.shape[1]} (oracle {int(fbr.sum())})")


def _centre_theta(faces):
    """All weights zero, b3 = exact shape function of a marker at a cell centre:
    the raw output is that phi for every marker (exact in float32)."""
    grid = oracle.Grid(faces, (True, True, True))
    h = [faces[d][1] - faces[d][0] for d in range(3)]
    centre = np.array([[faces[d][5] + 0.5 * h[d]] for d in range(3)])
    p = mlp.unflatten(np.zeros(mlp.N_PARAMS))
    p["b3"] = oracle.shape_exact(grid, centre, 1.0).phi[0].astype(np.float32)
    return mlp.flatten(p).astype(np.float32)


@pytest.mark.parametrize("thr", [0.2, 0.35, 0.45])
def test_raw_residual_gate_marker_by_marker(api, thr):
    """The gate reads the raw output's residual.  For the centre network on a
    uniform grid that residual is max_d |t_d| (t = offset from the cell centre in
    cell widths), so the fallback set is known in closed form; the GPU must fall
    back on exactly those markers (up to float32 rounding at the threshold),
    giving exact-MLS there and the projected centre phi elsewhere."""
    faces = [uniform_faces(16)] * 3
    grid = oracle.Grid(faces, (True, True, True))
    ctx = api.Context(faces, (True, True, True), real="f32", residual_max=thr)
    theta = _centre_theta(faces)
    ctx.surrogate_params(theta)
    rng = np.random.default_rng(int(thr * 100))
    x = np.stack([rng.uniform(faces[d][2], faces[d][14], size=3000) for d in range(3)]).astype(np.float32)
    area = np.full(3000, 1e-3, dtype=np.float32)
    g = run_gpu(ctx, x, area, "surrogate")
    sup = oracle.support(grid, x.astype(np.float64))
    t = np.stack([(x[d] - grid.faces[d][sup.home[d]]) / sup.hwidth[d] - 0.5 for d in range(3)])
    tmax = np.max(np.abs(t), axis=0)
    want = tmax > thr
    clear = np.abs(tmax - thr) > 1e-5                           # away from float32 rounding of the residual
    tr, fb = mlp.shape_surrogate(grid, x.astype(np.float64), theta.astype(np.float64), residual_max=thr)
    assert np.array_equal(fb[clear], want[clear])                 # the oracle agrees with the closed form
    ex = oracle.shape_exact(grid, x.astype(np.float64), 1.0).phi
    xi = np.stack([(sup.pos[d] - x[d][:, None]) / sup.hwidth[d][:, None] for d in range(3)])
    proj, _ = mlp.project(np.repeat(theta[None, -27:].astype(np.float64), 3000, axis=0), xi)
    d_ex = np.max(np.abs(g["phi"] - ex), axis=1)
    d_pr = np.max(np.abs(g["phi"] - proj), axis=1)
    got = d_ex < d_pr                                            # which of the two the GPU gave
    distinct = np.max(np.abs(ex - proj), axis=1) > 1e-4
    m = clear & distinct
    assert np.array_equal(got[m], want[m])
    assert np.all(np.minimum(d_ex, d_pr)[m] <= 1e-5)
    n_clear_fb = int(want[clear].sum())
    assert abs(g["status"]["surrogate_fallback"] - n_clear_fb) <= int((~clear).sum())
    assert 0 < want.sum() < len(want)



def test_surrogate_needs_parameters(api):
    faces, periodic = _grid()
    ctx = api.Context(faces, periodic, real="f32")
    from paper_1805_01113_gb300 import binding as B
    T = ctx.transfer(10)
    x = torch.zeros((3, 10), dtype=torch.float32, device=DEV)
    with pytest.raises(B.MlsError) as e:
        ctx.build_transfer(T, x, torch.ones(10, dtype=torch.float32, device=DEV), "surrogate")
    assert e.value.code == B.MLS_ERR_UNSUPPORTED
