"""Double-precision reference for exact-MLS and fast-MLS transfer functions.

TEST INFRASTRUCTURE ONLY (see the package docstring): the CUDA library never
imports, links or runs this file.

Notation follows Section 2 of the paper: a Lagrangian marker l at x_l, its
N_e = 27 Eulerian support nodes x_k (the centres of the home cell and of its
3x3x3 neighbourhood, Fig. 1a), the linear basis p = [1, x, y, z] (m = 4; the
quadratic m = 10 as an option), the
weight W(x_l - x_k), the moment matrix A (Eq. 3), the matrix B (Eq. 4), the
shape functions Phi^T = p^T(x_l) A^-1 B (Eq. 6), interpolation U = Phi^T u,
spreading f_k = sum_l c_l phi_k^l F_l with c_l from Eq. 8, and fast-MLS
(Eqs. 9-10: Shepard interpolation of exact shape functions tabulated on a
sub-Eulerian mesh of the home cell).

Readings of points the paper leaves open:
  * W is a Gaussian, W = exp(-r^2/eps^2), r measured per axis in units of the
    home cell's width (the paper only says the weight is a free choice).
  * Support nodes are cell centres; the home cell is the cell with
    face_i <= x < face_{i+1}; the support is home +/- 1 on each axis, wrapped
    on periodic axes and required to stay inside the grid on walled axes.
  * The sub-Eulerian mesh has n points per axis at -1/2 + i/(n-1) cell widths
    (faces included, so 3, 5, 9 points per axis as in Fig. 1b/1c).  In 3-D the
    Shepard sum runs over the 8 corners of the enclosing sub-cell, and the
    numerator of Eq. 10 is read as 1/d_i^2.
  * Node order inside a support: k = 9*(a_z+1) + 3*(a_y+1) + (a_x+1) for
    offsets a in {-1,0,1}^3 (x fastest); sub-node order s = (s_z*n + s_y)*n + s_x.
"""

from dataclasses import dataclass

import numpy as np

_A = np.array([-1, 0, 1])
# Offsets (a_x, a_y, a_z) of the 27 support nodes in the documented order.
NODE_OFFSETS = np.array([(ax, ay, az) for az in _A for ay in _A for ax in _A], dtype=np.int64)


class Grid:
    """Eulerian grid given by per-axis face coordinates (Section 2, Fig. 1a).

    Cell i of an axis spans [faces[i], faces[i+1]); its centre is the node used
    in the MLS support and its width enters Eqs. 7-8.
    """

    def __init__(self, faces, periodic):
        self.faces = [np.asarray(f, dtype=np.float64) for f in faces]
        self.periodic = tuple(bool(p) for p in periodic)
        self.n = tuple(len(f) - 1 for f in self.faces)
        self.centres = [0.5 * (f[:-1] + f[1:]) for f in self.faces]
        self.widths = [f[1:] - f[:-1] for f in self.faces]
        self.length = [f[-1] - f[0] for f in self.faces]
        for d in range(3):
            if self.n[d] < 3 or np.any(self.widths[d] <= 0):
                raise ValueError("each axis needs >= 3 cells with increasing faces")

    def uniform_axis(self, d, rtol=1e-12):
        w = self.widths[d]
        return bool(np.all(np.abs(w - w[0]) <= rtol * w[0]))


def marker_prep(vertices, tri, precision="f64"):
    """Marker positions and areas from a triangulated surface.

    The marker of a triangle is its centroid C = (V1 + V2 + V3)/3 (Section 3,
    description of Fig. 5a) and its area A_l is the triangle area used in the
    forcing volume Delta V_l = A_l h_l (text after Eq. 7).

    ``precision="f32"`` evaluates the same formulas in IEEE single precision in
    a fixed operation order, ((V1+V2)+V3)/3 and 0.5*sqrt((nx^2+ny^2)+nz^2),
    which is how the single-precision path stores its markers; the
    double-precision result stays the definition (a test bounds the gap).

    Returns (x (3, M), area (M,)).
    """
    dt = np.float64 if precision == "f64" else np.float32
    V = np.asarray(vertices).astype(dt)
    t = np.asarray(tri, dtype=np.int64)
    v1, v2, v3 = V[t[:, 0]], V[t[:, 1]], V[t[:, 2]]
    c = ((v1 + v2) + v3) / dt(3)
    e1 = v2 - v1
    e2 = v3 - v1
    nx = e1[:, 1] * e2[:, 2] - e1[:, 2] * e2[:, 1]
    ny = e1[:, 2] * e2[:, 0] - e1[:, 0] * e2[:, 2]
    nz = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
    area = dt(0.5) * np.sqrt((nx * nx + ny * ny) + nz * nz)
    return np.ascontiguousarray(c.T), area


def locate(grid, x):
    """Home cell of each marker (Section 2: the cell that contains the marker).

    Returns (home (3, M) int64, ok (M,) bool).  ok is False for non-finite
    positions, positions outside [faces[0], faces[-1]), and, on a walled
    (non-periodic) axis, home cells whose 3-wide support would leave the grid.
    """
    x = np.asarray(x, dtype=np.float64)
    M = x.shape[1]
    home = np.zeros((3, M), dtype=np.int64)
    ok = np.all(np.isfinite(x), axis=0)
    for d in range(3):
        xd = np.where(np.isfinite(x[d]), x[d], grid.faces[d][0] - 1.0)
        i = np.searchsorted(grid.faces[d], xd, side="right") - 1
        inside = (i >= 0) & (i < grid.n[d])
        if not grid.periodic[d]:
            inside &= (i >= 1) & (i <= grid.n[d] - 2)
        ok &= inside
        home[d] = np.clip(i, 0, grid.n[d] - 1)
    return home, ok


@dataclass
class Support:
    """The 27-node support of each marker (Fig. 1a)."""
    home: np.ndarray     # (3, M) home cell
    ok: np.ndarray       # (M,) marker usable
    idx: np.ndarray      # (3, M, 27) wrapped node cell indices
    pos: np.ndarray      # (3, M, 27) node coordinates (periodic images unwrapped)
    width: np.ndarray    # (3, M, 27) widths of the node cells
    hwidth: np.ndarray   # (3, M) widths of the home cell


def support(grid, x, home=None):
    """Support nodes = centres of the home cell and its 26 neighbours (Fig. 1a caption)."""
    if home is None:
        home, ok = locate(grid, x)
    else:
        home = np.asarray(home, dtype=np.int64)
        ok = np.all(np.isfinite(x), axis=0)
    M = home.shape[1]
    idx = np.empty((3, M, 27), dtype=np.int64)
    pos = np.empty((3, M, 27))
    width = np.empty((3, M, 27))
    hwidth = np.empty((3, M))
    for d in range(3):
        n = grid.n[d]
        j = home[d][:, None] + NODE_OFFSETS[None, :, d]
        if grid.periodic[d]:
            jw = np.mod(j, n)
            shift = np.where(j < 0, -grid.length[d], np.where(j >= n, grid.length[d], 0.0))
        else:
            jw = np.clip(j, 0, n - 1)
            shift = np.zeros(j.shape)
        idx[d] = jw
        pos[d] = grid.centres[d][jw] + shift
        width[d] = grid.widths[d][jw]
        hwidth[d] = grid.widths[d][home[d]]
    return Support(home, ok, idx, pos, width, hwidth)


def gaussian_weight(x, sup, eps):
    """W(x_l - x_k) = exp(-r^2/eps^2), r^2 = sum_d ((x_k,d - x_l,d)/Delta_d^home)^2.

    The paper leaves W open (text after Eq. 2: exponential or spline weights);
    this Gaussian, untruncated over the 27 nodes, is the reading used here.
    """
    r2 = np.zeros(sup.pos.shape[1:])
    for d in range(3):
        r2 += ((sup.pos[d] - x[d][:, None]) / sup.hwidth[d][:, None]) ** 2
    return np.exp(-r2 / eps ** 2)


@dataclass
class Transfer:
    phi: np.ndarray      # (M, 27) shape functions; zero rows for unusable markers
    sup: Support


def basis_values(xi, m=4):
    """Basis vector p of Section 2 (text after Eq. 2) at the points xi (3, ...).

    The terms come from Pascal's pyramid: m = 4 is the linear basis
    [1, x, y, z] the paper uses; m = 10 adds the six degree-2 terms
    [x^2, y^2, z^2, xy, yz, zx] (the paper allows any m; fast-MLS does not
    depend on it).  Returns an array of shape xi.shape[1:] + (m,).
    """
    if m not in (4, 10):
        raise ValueError("basis size m must be 4 or 10")
    x, y, z = xi[0], xi[1], xi[2]
    cols = [np.ones_like(x), x, y, z]
    if m == 10:
        cols += [x * x, y * y, z * z, x * y, y * z, z * x]
    return np.stack(cols, axis=-1)


def shape_exact(grid, x, eps=1.0, home=None, basis=4):
    """Exact-MLS shape functions, Eqs. 3, 4 and 6.

    The basis is written in marker-centred, home-width-scaled coordinates,
    p~(x) = p((x - x_l)/Delta^home), an invertible affine change of the
    paper's coordinates that maps the space spanned by p (linear, m = 4, or
    quadratic, m = 10; see basis_values) onto itself and so leaves Phi
    unchanged, with p~(x_l) = e_0.
    A(x_l) = sum_k W_k p~(x_k) p~(x_k)^T (Eq. 3), B = [W_k p~(x_k)] (Eq. 4),
    Phi^T = p~(x_l)^T A^-1 B (Eq. 6), solved with a library dense solve.
    """
    x = np.asarray(x, dtype=np.float64)
    sup = support(grid, x, home)
    W = gaussian_weight(x, sup, eps)                       # (M, 27)
    M = x.shape[1]
    xi = np.stack([(sup.pos[d] - x[d][:, None]) / sup.hwidth[d][:, None] for d in range(3)])
    P = basis_values(xi, basis)                            # (M, 27, m)
    A = np.einsum("mk,mki,mkj->mij", W, P, P)              # Eq. 3
    B = np.transpose(W[:, :, None] * P, (0, 2, 1))         # Eq. 4, (M, m, 27)
    good = sup.ok.copy()
    phi = np.zeros((M, 27))
    if np.any(good):
        X = np.linalg.solve(A[good], B[good])              # A^-1 B
        pl = basis_values(np.zeros(3), basis)              # p~(x_l) = e_0
        phi[good] = np.einsum("i,mik->mk", pl, X)          # Eq. 6
    return Transfer(phi, sup)


def moment_matrix(grid, x, eps=1.0, home=None, basis=4):
    """The moment matrix A(x_l) of Eq. 3 in the marker-centred, home-width-scaled
    basis of shape_exact, (M, m, m); and its 1-norm condition number
    ||A||_1 ||A^-1||_1 (the quantity the single-precision solve is gated on),
    (M,), infinite where A is singular or the marker has no support."""
    x = np.asarray(x, dtype=np.float64)
    sup = support(grid, x, home)
    W = gaussian_weight(x, sup, eps)
    xi = np.stack([(sup.pos[d] - x[d][:, None]) / sup.hwidth[d][:, None] for d in range(3)])
    P = basis_values(xi, basis)
    A = np.einsum("mk,mki,mkj->mij", W, P, P)
    cond = np.full(x.shape[1], np.inf)
    for m in np.nonzero(sup.ok)[0]:
        try:
            cond[m] = np.linalg.norm(A[m], 1) * np.linalg.norm(np.linalg.inv(A[m]), 1)
        except np.linalg.LinAlgError:
            pass
    return A, cond


def shape_exact_gradient(grid, x, eps=1.0, home=None):
    """Spatial derivatives of the exact-MLS shape functions at the markers.

    The paper uses MLS also for velocity and pressure gradients at the marker
    (Section 2: derivatives of the interpolated field); the derivative of
    Eq. 6 with respect to the evaluation point x follows from the product
    rule.  With the basis centred at a fixed c = x_l,
    p~(y) = [1, (y - c)/Delta^home], A(x) = sum_j W_j(x) p~_j p~_j^T (Eq. 3)
    and gamma = A^-1 p~(x):
        d_d phi_k = d_d W_k p~_k^T gamma + W_k p~_k^T A^-1 (d_d p~ - d_d A gamma),
    d_d A = sum_j d_d W_j p~_j p~_j^T, d_d p~ = e_{d+1}/Delta_d, and for the
    Gaussian d_d W_j = W_j 2 (x_j,d - x_d) / (eps Delta_d)^2.  The home cell
    (and so the support and the width scaling) is held fixed.

    Returns dphi (M, 3, 27), zero rows for unusable markers.
    """
    x = np.asarray(x, dtype=np.float64)
    sup = support(grid, x, home)
    W = gaussian_weight(x, sup, eps)                       # (M, 27)
    M = x.shape[1]
    P = np.ones((M, 27, 4))
    for d in range(3):
        P[:, :, d + 1] = (sup.pos[d] - x[d][:, None]) / sup.hwidth[d][:, None]
    A = np.einsum("mk,mki,mkj->mij", W, P, P)
    dphi = np.zeros((M, 3, 27))
    good = sup.ok
    if not np.any(good):
        return dphi
    Ag, Wg, Pg = A[good], W[good], P[good]
    pl = np.zeros((Ag.shape[0], 4))
    pl[:, 0] = 1.0
    gamma = np.linalg.solve(Ag, pl[:, :, None])[:, :, 0]   # A^-1 p~(x_l)
    out = np.zeros((Ag.shape[0], 3, 27))
    for d in range(3):
        hd = sup.hwidth[d][good][:, None]
        dW = Wg * 2.0 * (sup.pos[d][good] - x[d][good][:, None]) / (eps * hd) ** 2
        dA = np.einsum("mk,mki,mkj->mij", dW, Pg, Pg)
        dp = np.zeros((Ag.shape[0], 4))
        dp[:, d + 1] = 1.0 / hd[:, 0]
        rhs = dp - np.einsum("mij,mj->mi", dA, gamma)
        dgamma = np.linalg.solve(Ag, rhs[:, :, None])[:, :, 0]
        out[:, d] = dW * np.einsum("mki,mi->mk", Pg, gamma) + Wg * np.einsum("mki,mi->mk", Pg, dgamma)
    dphi[good] = out
    return dphi


def interpolate_gradient(dphi, sup, u):
    """Velocity gradient at the markers: G[c, d, l] = sum_k d_d phi_k^l u_c,k."""
    ix, iy, iz = sup.idx
    G = np.empty((3, 3, dphi.shape[0]))
    for c in range(3):
        uk = u[c][iz, iy, ix]                              # (M, 27)
        for d in range(3):
            G[c, d] = np.sum(dphi[:, d] * uk, axis=1)
    return G


def shape_exact_absolute_basis(grid, x, eps=1.0, home=None):
    """Eqs. 3, 4, 6 exactly as printed, with p = [1, x, y, z] in absolute coordinates.

    Mathematically identical to :func:`shape_exact`; used as a cross-check of
    the centred form (it is badly conditioned on fine grids, so only small
    cases use it).
    """
    x = np.asarray(x, dtype=np.float64)
    sup = support(grid, x, home)
    W = gaussian_weight(x, sup, eps)
    M = x.shape[1]
    P = np.ones((M, 27, 4))
    for d in range(3):
        P[:, :, d + 1] = sup.pos[d]
    A = np.einsum("mk,mki,mkj->mij", W, P, P)
    B = np.transpose(W[:, :, None] * P, (0, 2, 1))
    pl = np.concatenate([np.ones((M, 1)), x.T], axis=1)    # p(x_l)
    phi = np.zeros((M, 27))
    good = sup.ok
    if np.any(good):
        X = np.linalg.solve(A[good], B[good])
        phi[good] = np.einsum("mi,mik->mk", pl[good], X)
    return Transfer(phi, sup)


def subnode_offsets(n_sub):
    """Sub-Eulerian mesh points per axis, in home-cell units: -1/2 + i/(n-1) (Fig. 1b/1c)."""
    return -0.5 + np.arange(n_sub, dtype=np.float64) / (n_sub - 1)


def fast_table(grid, home, n_sub=9, eps=1.0, basis=4):
    """Exact shape functions at the n^3 sub-Eulerian nodes of one home cell (Section 2, Fig. 1b/1c).

    ``home`` is a length-3 cell index.  Returns (n^3, 27) in sub-node order
    s = (s_z*n + s_y)*n + s_x.  Nodes on the cell faces keep this home cell's
    support (the home index is forced rather than re-located).
    """
    off = subnode_offsets(n_sub)
    sz, sy, sx = np.meshgrid(off, off, off, indexing="ij")
    rel = [sx.ravel(), sy.ravel(), sz.ravel()]
    X = np.empty((3, n_sub ** 3))
    for d in range(3):
        X[d] = grid.faces[d][home[d]] + (rel[d] + 0.5) * grid.widths[d][home[d]]
    H = np.repeat(np.asarray(home, dtype=np.int64)[:, None], n_sub ** 3, axis=1)
    return shape_exact(grid, X, eps, home=H, basis=basis).phi


def _table_key(grid, home):
    # On a uniform axis every cell has the same table (Section 2: markers at the
    # same relative position get the same shape functions); use the middle cell.
    return tuple(int(home[d]) if not grid.uniform_axis(d) else grid.n[d] // 2 for d in range(3))


def shape_fast(grid, x, eps=1.0, n_sub=9, home=None, subcell=None, tables=None, basis=4):
    """Fast-MLS shape functions, Eqs. 9-10.

    The marker's offset in its home cell, t in [-1/2, 1/2)^3, selects the
    enclosing sub-cell of the sub-Eulerian mesh; its 8 corners i carry tabulated
    exact shape functions Phi_e^i; with d_i the marker-to-corner distance in
    home-cell units, alpha_i = (1/d_i^2) / sum_j (1/d_j^2) and
    Phi_f = sum_i alpha_i Phi_e^i.  A marker within 1e-12 of a corner takes that
    corner's Phi_e.

    ``subcell`` (3, M) optionally forces the sub-cell (used to compare with a
    single-precision caller that resolved a sub-cell face the other way).
    ``tables`` is an optional dict cache shared between calls.  ``basis``
    (m = 4 or 10) is the basis of the tabulated exact shape functions.
    """
    x = np.asarray(x, dtype=np.float64)
    sup = support(grid, x, home)
    M = x.shape[1]
    nm1 = n_sub - 1
    t = np.empty((3, M))
    for d in range(3):
        t[d] = (x[d] - grid.faces[d][sup.home[d]]) / sup.hwidth[d] - 0.5
    u = np.where(sup.ok, (t + 0.5) * nm1, 0.0)
    if subcell is None:
        s = np.minimum(np.floor(u), nm1 - 1).astype(np.int64)
    else:
        s = np.asarray(subcell, dtype=np.int64)
    lam = u - s
    tables = {} if tables is None else tables
    phi = np.zeros((M, 27))
    corners = [(cx, cy, cz) for cz in (0, 1) for cy in (0, 1) for cx in (0, 1)]
    for m in np.nonzero(sup.ok)[0]:
        key = _table_key(grid, sup.home[:, m])
        if (key, basis) not in tables:
            tables[(key, basis)] = fast_table(grid, key, n_sub, eps, basis)
        T = tables[(key, basis)]
        d2 = np.array([sum(((lam[d, m] - c[d]) / nm1) ** 2 for d in range(3)) for c in corners])
        nodes = [((s[2, m] + c[2]) * n_sub + (s[1, m] + c[1])) * n_sub + (s[0, m] + c[0]) for c in corners]
        if np.min(d2) < 1e-24:
            phi[m] = T[nodes[int(np.argmin(d2))]]
        else:
            inv = 1.0 / d2
            alpha = inv / np.sum(inv)                      # Eq. 10
            phi[m] = alpha @ T[nodes]                      # Eq. 9
    return Transfer(phi, sup)


def forcing_scale(tr, area):
    """Scaling factor c_l of Eq. 8.

    h_l = sum_k phi_k (Dx_k + Dy_k + Dz_k)/3, Delta V_l = A_l h_l (text after
    Eq. 7), c_l = Delta V_l / sum_k phi_k Delta V_k with Delta V_k the node
    cell's volume.  Unusable markers get c_l = 0.
    """
    w = tr.sup.width
    h = np.sum(tr.phi * (w[0] + w[1] + w[2]), axis=1) / 3.0
    dVl = np.asarray(area, dtype=np.float64) * h
    den = np.sum(tr.phi * (w[0] * w[1] * w[2]), axis=1)
    c = np.zeros_like(dVl)
    good = tr.sup.ok & (den != 0)
    c[good] = dVl[good] / den[good]
    return c


def interpolate(tr, u):
    """Euler-to-Lagrange interpolation U_l = Phi^T u (Section 2, text after Eq. 6).

    u is (3, nz, ny, nx); returns U (3, M).
    """
    ix, iy, iz = tr.sup.idx
    U = np.empty((3, tr.phi.shape[0]))
    for c in range(3):
        U[c] = np.sum(tr.phi * u[c][iz, iy, ix], axis=1)
    return U


@dataclass
class SparseField:
    """Cells touched by spreading: linear index (iz*ny + iy)*nx + ix and values (3, K)."""
    keys: np.ndarray
    values: np.ndarray

    def to_dense(self, n):
        nx, ny, nz = n
        f = np.zeros((3, nz * ny * nx))
        f[:, self.keys] = self.values
        return f.reshape(3, nz, ny, nx)


def spread(tr, c, F, n):
    """Lagrange-to-Euler spreading f_k = sum_l c_l phi_k^l F_l (text after Eq. 7).

    F is (3, M); ``n`` = (nx, ny, nz).  Accumulates in double precision into a
    sparse map of the touched cells.
    """
    nx, ny, nz = n
    good = tr.sup.ok
    ix, iy, iz = (a[good] for a in tr.sup.idx)
    keys = ((iz * ny + iy) * nx + ix).ravel()
    uk, inv = np.unique(keys, return_inverse=True)
    w = tr.phi[good] * np.asarray(c, dtype=np.float64)[good][:, None]   # c_l phi_k^l
    vals = np.empty((3, len(uk)))
    for comp in range(3):
        contrib = (w * np.asarray(F[comp], dtype=np.float64)[good][:, None]).ravel()
        vals[comp] = np.bincount(inv.ravel(), weights=contrib, minlength=len(uk))
    return SparseField(uk, vals)


def direct_forcing(tr, c, u, Vb, dt, n):
    """One direct-forcing transfer (Section 2, text after Eq. 6 and Eq. 7).

    U_l = Phi^T u (interpolated velocity), F_l = (V_b,l - U_l) / dt (the IBM
    force that drives the fluid velocity at the marker to the desired V_b),
    then f_k = sum_l c_l phi_k^l F_l.  Markers without a usable support get
    U_l = 0 and F_l = 0 (no forcing).  Returns (U, F, SparseField).
    """
    U = interpolate(tr, u)
    U[:, ~tr.sup.ok] = 0.0
    F = (np.asarray(Vb, dtype=np.float64) - U) / dt
    F[:, ~tr.sup.ok] = 0.0
    return U, F, spread(tr, c, F, n)
