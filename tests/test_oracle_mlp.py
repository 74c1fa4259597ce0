"""Pins for the surrogate oracle (network, backpropagation, Adam, projection, generator)."""

import numpy as np

import oracle
from oracle import mlp
from workloads import tanh_faces, uniform_faces

RNG = np.random.default_rng(31)


def test_splitmix64_published_values():
    # First outputs of splitmix64 started from state 0 (Vigna's reference implementation).
    got = [int(v) for v in mlp.splitmix64(np.arange(3), 0)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = mlp.uniform01(np.arange(100000), 12345)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005
    assert np.all(u * 2 ** 24 == np.floor(u * 2 ** 24))      # float32-exact


def test_backprop_matches_central_differences():
    theta = mlp.init_params(7) + 0.05 * RNG.normal(size=mlp.N_PARAMS)
    X = RNG.normal(size=(9, mlp.N_IN))
    T = RNG.normal(size=(9, mlp.N_OUT)) * 0.1
    L, g = mlp.loss_and_grad(theta, X, T)
    idx = RNG.choice(mlp.N_PARAMS, size=60, replace=False)
    h = 1e-6
    for q in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[q] = h
        fd = (mlp.loss_and_grad(theta + e, X, T)[0] - mlp.loss_and_grad(theta - e, X, T)[0]) / (2 * h)
        assert abs(fd - g[q]) <= 1e-7 * max(1.0, abs(g[q])) + 1e-10


def test_network_special_cases():
    theta = np.zeros(mlp.N_PARAMS)
    p = mlp.unflatten(theta)
    p["b3"] = np.arange(27.0)
    Y, _ = mlp.forward(mlp.flatten(p), RNG.normal(size=(4, 6)))
    assert np.all(Y == np.arange(27.0))                      # zero weights: output = b3
    # One hidden path: y_0 = w3 * tanh(w2 * tanh(w1 x_0 + b1) + b2) + b3.
    p = mlp.unflatten(np.zeros(mlp.N_PARAMS))
    p["W1"][0, 0], p["b1"][0], p["W2"][0, 0], p["b2"][0], p["W3"][0, 0], p["b3"][0] = 0.7, 0.1, -1.3, 0.2, 2.0, 0.5
    x = np.array([[0.4, 9, 9, 9, 9, 9]])
    Y, _ = mlp.forward(mlp.flatten(p), x)
    assert abs(Y[0, 0] - (2.0 * np.tanh(-1.3 * np.tanh(0.7 * 0.4 + 0.1) + 0.2) + 0.5)) < 1e-15


def test_adam_first_step_is_signed_learning_rate():
    theta = np.zeros(5)
    g = np.array([3.0, -0.2, 1e-3, 0.0, -7.0])
    th, m, v = mlp.adam_step(theta, g, np.zeros(5), np.zeros(5), 1, 0.01)
    # m_hat = g, v_hat = g^2 after bias correction: step = lr * g / (|g| + eps).
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_init_is_glorot_uniform():
    theta = mlp.init_params(99)
    p = mlp.unflatten(theta)
    for name, (fo, fi) in (("W1", (64, 6)), ("W2", (64, 64)), ("W3", (27, 64))):
        a = np.sqrt(6.0 / (fi + fo))
        assert np.max(np.abs(p[name])) <= a and np.max(np.abs(p[name])) > 0.8 * a
    assert np.all(p["b1"] == 0) and np.all(p["b2"] == 0) and np.all(p["b3"] == 0)


def _grid():
    return oracle.Grid([uniform_faces(24), uniform_faces(24), tanh_faces(24, 1.5)], (True, True, False))


def _markers(grid, m):
    x = np.empty((3, m))
    for d in range(3):
        f = grid.faces[d]
        x[d] = RNG.uniform(f[2], f[grid.n[d] - 2], size=m)
    return x


def test_projection_properties():
    grid = _grid()
    x = _markers(grid, 50)
    tr = oracle.shape_exact(grid, x, 1.0)
    xi = np.stack([(tr.sup.pos[d] - x[d][:, None]) / tr.sup.hwidth[d][:, None] for d in range(3)])
    # Exact MLS already satisfies the constraints: projection leaves it unchanged.
    pe, r = mlp.project(tr.phi, xi)
    assert np.max(np.abs(r)) < 1e-12 and np.max(np.abs(pe - tr.phi)) < 1e-12
    # A perturbed phi is mapped onto the constraints, closer to exact, idempotently.
    noisy = tr.phi + 1e-3 * RNG.normal(size=tr.phi.shape)
    pn, _ = mlp.project(noisy, xi)
    assert np.max(mlp.reproduction_residual(pn, xi)) < 1e-13
    assert np.all(np.linalg.norm(pn - tr.phi, axis=1) <= np.linalg.norm(noisy - tr.phi, axis=1) + 1e-15)
    pp, _ = mlp.project(pn, xi)
    assert np.max(np.abs(pp - pn)) < 1e-13


def test_features():
    g = oracle.Grid([uniform_faces(8)] * 3, (True, True, True))
    home = np.array([[1, 2], [3, 4], [5, 6]])
    X = mlp.features(g, home, np.array([[0.1, -0.2], [0.3, 0.0], [-0.4, 0.25]]))
    assert np.all(X[:, 3:] == 0) and np.allclose(X[:, :3], [[0.1, 0.3, -0.4], [-0.2, 0.0, 0.25]])
    faces = [uniform_faces(8), uniform_faces(8), np.array([0, 1, 3, 6, 10, 15, 21, 28, 36.0]) / 18 - 1]
    g = oracle.Grid(faces, (True, True, False))
    X = mlp.features(g, np.array([[0], [0], [3]]), np.zeros((3, 1)))
    # widths along z: 1, 2, 3, 4, ... (/18); home 3 has 4, neighbours 3 and 5; x width 2/8.
    assert np.allclose(X[0, 3:], [np.log(3 / 4), np.log(5 / 4), np.log((4 / 18) / 0.25)])


def test_surrogate_fallback_paths():
    grid = _grid()
    x = _markers(grid, 40)
    ex = oracle.shape_exact(grid, x, 1.0).phi
    # Non-finite network output: every marker falls back to exact MLS.
    bad = np.full(mlp.N_PARAMS, np.nan)
    tr, fb = mlp.shape_surrogate(grid, x, bad)
    assert fb.all() and np.max(np.abs(tr.phi - ex)) < 1e-14
    # Zero network: the raw output 0 has residual |sum phi - 1| = 1, so every
    # marker falls back at the default threshold; above 1 none does, and the
    # projection gives the minimum-norm reproducing phi.
    tr, fb = mlp.shape_surrogate(grid, x, np.zeros(mlp.N_PARAMS))
    assert fb.all() and np.max(np.abs(tr.phi - ex)) < 1e-14
    tr, fb = mlp.shape_surrogate(grid, x, np.zeros(mlp.N_PARAMS), residual_max=1.0 + 1e-9)
    assert not fb.any()
    assert np.max(np.abs(tr.phi.sum(1) - 1)) < 1e-13


def centre_network(grid):
    """Parameters whose output is the exact shape function of a marker at the
    centre of a uniform cell, whatever the input (all weights zero, b3 = phi)."""
    h = [grid.faces[d][1] - grid.faces[d][0] for d in range(3)]
    centre = np.array([[grid.faces[d][5] + 0.5 * h[d]] for d in range(3)])
    p = mlp.unflatten(np.zeros(mlp.N_PARAMS))
    p["b3"] = oracle.shape_exact(grid, centre, 1.0).phi[0]
    return mlp.flatten(p)


def test_raw_residual_gate_closed_form():
    """The gate reads the raw output.  For the centre network on a uniform grid
    the raw residual is max_d |t_d| (t = offset from the cell centre in cell
    widths): phi_c sums to 1 and reproduces the centre, so sum_k phi_c,k xi_k,d
    = -t_d.  Markers fall back exactly where max_d |t_d| > threshold."""
    grid = oracle.Grid([uniform_faces(16)] * 3, (True, True, True))
    theta = centre_network(grid)
    x = _markers(grid, 400)
    sup = oracle.support(grid, x)
    t = np.stack([(x[d] - grid.faces[d][sup.home[d]]) / sup.hwidth[d] - 0.5 for d in range(3)])
    tmax = np.max(np.abs(t), axis=0)
    ex = oracle.shape_exact(grid, x, 1.0).phi
    for thr in (0.2, 0.35, 0.45):
        tr, fb = mlp.shape_surrogate(grid, x, theta, residual_max=thr)
        assert np.array_equal(fb, tmax > thr)
        assert np.max(np.abs(tr.phi[fb] - ex[fb])) < 1e-14
        # accepted markers: the projection of phi_c, which reproduces linear fields at x
        acc = ~fb
        xi = np.stack([(sup.pos[d][acc] - x[d][acc, None]) / sup.hwidth[d][acc, None] for d in range(3)])
        assert np.max(mlp.reproduction_residual(tr.phi[acc], xi)) < 1e-13
        assert np.max(np.abs(tr.phi[acc] - ex[acc])) < 1.0        # not exact-MLS, only reproducing
    # Half-way threshold splits the markers in two non-empty sets.
    _, fb = mlp.shape_surrogate(grid, x, theta, residual_max=0.35)
    assert 0 < fb.sum() < len(fb)
