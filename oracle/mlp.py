"""Double-precision reference for the learned shape-function surrogate.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no learned component; this follows the surrogate form that sits
on top of exact-MLS: on a grid uniform in all but one axis, the shape functions
of a marker depend only on its offset t in the home cell and the width ratios
of the non-uniform axis (Section 2, premise of fast-MLS), so a small network
can map those to the 27 values.

Readings:
  * features (6): t_x, t_y, t_z, ln(D_{i-1}/D_i), ln(D_{i+1}/D_i), ln(D_i/D_u)
    with D the widths along the non-uniform axis (z when all are uniform, then
    the three ratio features are 0) and D_u the width of the first other axis;
  * network: 6 -> 64 -> 64 -> 27, tanh hidden activations, linear output,
    parameters stored flat as W1[64][6], b1[64], W2[64][64], b2[64],
    W3[27][64], b3[27];
  * loss: mean squared error over the 27 outputs and the batch; Adam with
    beta1 = 0.9, beta2 = 0.999, eps = 1e-8;
  * the gate: a marker whose raw network output has a linear-reproduction
    residual max(|sum_k phi_k - 1|, |sum_k phi_k xi_k,d|) above the threshold
    (or not finite) takes the exact-MLS value (reproduction of linear fields
    is the property MLS guarantees, Section 2); an accepted output is then
    projected orthogonally onto the affine set {sum_k phi_k = 1,
    sum_k phi_k xi_k = 0};
  * random draws use the splitmix64 finaliser (Steele, Lea & Flood 2014;
    constants as published by Vigna) as a counter-based generator.
"""

import numpy as np

from . import mls as _mls

N_IN, N_H, N_OUT = 6, 64, 27
SIZES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
         ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter, seed):
    """z = seed + (counter + 1) * golden; then the splitmix64 output mix."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(counter, seed):
    """float32-exact uniform numbers in [0, 1): top 24 bits of the draw times 2^-24."""
    return (splitmix64(counter, seed) >> np.uint64(40)).astype(np.float64) * 2.0 ** -24


def unflatten(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def init_params(seed):
    """Glorot-uniform weights, zero biases; draw q of the flat vector is counter q."""
    theta = np.zeros(N_PARAMS)
    o = 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        if name.startswith("W"):
            fan_out, fan_in = shape
            a = np.sqrt(6.0 / (fan_in + fan_out))
            theta[o:o + n] = (2.0 * uniform01(np.arange(o, o + n), seed) - 1.0) * a
        o += n
    return theta


def class_axis(grid):
    nonuni = [d for d in range(3) if not grid.uniform_axis(d)]
    if len(nonuni) > 1:
        raise ValueError("the surrogate needs at most one non-uniform axis")
    return nonuni[0] if nonuni else 2


def features(grid, home, t):
    """Network inputs (M, 6) for markers with home cells (3, M) and offsets t (3, M)."""
    c = class_axis(grid)
    u = 0 if c != 0 else 1
    n = grid.n[c]
    w = grid.widths[c]
    i = home[c]
    if grid.periodic[c]:
        im, ip = np.mod(i - 1, n), np.mod(i + 1, n)
    else:
        im, ip = np.clip(i - 1, 0, n - 1), np.clip(i + 1, 0, n - 1)
    X = np.empty((home.shape[1], N_IN))
    X[:, 0:3] = np.asarray(t, dtype=np.float64).T
    X[:, 3] = np.log(w[im] / w[i])
    X[:, 4] = np.log(w[ip] / w[i])
    X[:, 5] = np.log(w[i] / grid.widths[u][0])
    return X


def forward(theta, X):
    """Returns (Y (B, 27), cache) for the 6-64-64-27 tanh network."""
    p = unflatten(theta)
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = np.tanh(Z1)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = np.tanh(Z2)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, (X, H1, H2)


def loss_and_grad(theta, X, T):
    """Mean squared error over outputs and batch, and its gradient (backpropagation)."""
    p = unflatten(theta)
    Y, (X, H1, H2) = forward(theta, X)
    B = X.shape[0]
    R = Y - T
    L = float(np.sum(R * R) / (B * N_OUT))
    dY = 2.0 * R / (B * N_OUT)
    g = {"W3": dY.T @ H2, "b3": dY.sum(0)}
    dZ2 = (dY @ p["W3"]) * (1.0 - H2 * H2)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(0)
    dZ1 = (dZ2 @ p["W2"]) * (1.0 - H1 * H1)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(0)
    return L, flatten(g)


def adam_step(theta, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected); `step` counts from 1.  Returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def project(phi, xi):
    """Orthogonal projection of phi (M, 27) onto {sum phi = 1, sum phi xi_d = 0}.

    xi (3, M, 27) are the node offsets in home-cell units.  Returns (phi', r)
    with r (M, 4) the constraint residual of the input.
    """
    M = phi.shape[0]
    P = np.ones((M, 27, 4))
    for d in range(3):
        P[:, :, d + 1] = xi[d]
    r = np.einsum("mk,mki->mi", phi, P) - np.array([1.0, 0.0, 0.0, 0.0])
    G = np.einsum("mki,mkj->mij", P, P)
    lam = np.linalg.solve(G, r[:, :, None])[:, :, 0]
    return phi - np.einsum("mki,mi->mk", P, lam), r


def reproduction_residual(phi, xi):
    """max(|sum phi - 1|, |sum phi xi_d|) per marker."""
    r = np.abs(np.sum(phi, axis=1) - 1.0)
    for d in range(3):
        r = np.maximum(r, np.abs(np.sum(phi * xi[d], axis=1)))
    return r


def shape_surrogate(grid, x, theta, eps=1.0, residual_max=1e-4, home=None):
    """Surrogate shape functions with exact-MLS fallback.

    Returns (Transfer, used_fallback (M,) bool).  Network evaluation is in
    double precision here; the GPU evaluates it with bfloat16 operands.
    """
    x = np.asarray(x, dtype=np.float64)
    sup = _mls.support(grid, x, home)
    t = np.empty((3, x.shape[1]))
    xi = np.empty((3, x.shape[1], 27))
    for d in range(3):
        t[d] = (x[d] - grid.faces[d][sup.home[d]]) / sup.hwidth[d] - 0.5
        xi[d] = (sup.pos[d] - x[d][:, None]) / sup.hwidth[d][:, None]
    Y, _ = forward(theta, features(grid, sup.home, t))
    res = reproduction_residual(Y, xi)               # the raw output, before projection
    phi, _ = project(Y, xi)
    bad = ~(res <= residual_max) | ~np.all(np.isfinite(phi), axis=1)
    bad &= sup.ok
    if np.any(bad):
        phi[bad] = _mls.shape_exact(grid, x[:, bad], eps, home=sup.home[:, bad]).phi
    phi[~sup.ok] = 0.0
    return _mls.Transfer(phi, sup), bad


def training_samples(grid, first, count, seed, eps=1.0):
    """Training inputs and exact-MLS labels for samples first .. first+count-1.

    Sample s uses counters 4s, 4s+1, 4s+2 for the offsets t_d = u - 1/2 and
    counter 4s+3 for the home index along the non-uniform axis: with z the
    draw, lo + floor((z >> 32) * range / 2^32) over the usable cells (1 .. n-2
    on a walled axis, 0 .. n-1 on a periodic one).  The other axes use their
    middle cell.  Labels are exact-MLS shape functions (Eqs. 3-6) at the
    resulting position.  Returns (X (count, 6), phi (count, 27)).
    """
    c = class_axis(grid)
    s = np.arange(first, first + count, dtype=np.uint64)
    t = np.stack([uniform01(np.uint64(4) * s + np.uint64(q), seed) - 0.5 for q in range(3)])
    z = splitmix64(np.uint64(4) * s + np.uint64(3), seed)
    n = grid.n[c]
    lo, hi = (0, n - 1) if grid.periodic[c] else (1, n - 2)
    span = np.uint64(hi - lo + 1)
    cls = lo + (((z >> np.uint64(32)) * span) >> np.uint64(32)).astype(np.int64)
    home = np.empty((3, count), dtype=np.int64)
    for d in range(3):
        home[d] = cls if d == c else grid.n[d] // 2
    X = features(grid, home, t)
    x = np.empty((3, count))
    for d in range(3):
        x[d] = grid.faces[d][home[d]] + (t[d] + 0.5) * grid.widths[d][home[d]]
    return X, _mls.shape_exact(grid, x, eps, home=home).phi
