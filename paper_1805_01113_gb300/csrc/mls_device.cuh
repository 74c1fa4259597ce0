// Device-side building blocks of the MLS transfer library: grid description,
// home-cell location, per-axis support geometry and the two shape-function
// evaluations (exact-MLS, Eqs. 3-6; fast-MLS, Eqs. 9-10).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace mls {

// One grid axis.  Cell i spans [faces[i], faces[i+1]); `uniform` axes also
// carry lo and h so the home cell comes from one multiply plus a face check.
// IEEE operations rounded to nearest with no contraction, so that a fixed
// order of operations is reproducible bit for bit by any IEEE implementation.
template <typename R> struct Ops;
template <> struct Ops<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
  static __device__ __forceinline__ float sqrt_(float a) { return __fsqrt_rn(a); }
  static __device__ __forceinline__ float nan_() { return __int_as_float(0x7fc00000); }
};
template <> struct Ops<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
  static __device__ __forceinline__ double sqrt_(double a) { return __dsqrt_rn(a); }
  static __device__ __forceinline__ double nan_() { return __longlong_as_double(0x7ff8000000000000ULL); }
};

// Marker of a triangle (Section 3): centroid C = ((V1+V2)+V3)/3 and area
// |(V2-V1)x(V3-V1)|/2, in this order of operations.
template <typename R>
__device__ __forceinline__ void triangle_marker(const R a[3], const R b[3], const R c[3], R x[3], R& area) {
  using O = Ops<R>;
  R e1[3], e2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    x[d] = O::div(O::add(O::add(a[d], b[d]), c[d]), R(3));
    e1[d] = O::sub(b[d], a[d]);
    e2[d] = O::sub(c[d], a[d]);
  }
  const R nx = O::sub(O::mul(e1[1], e2[2]), O::mul(e1[2], e2[1]));
  const R ny = O::sub(O::mul(e1[2], e2[0]), O::mul(e1[0], e2[2]));
  const R nz = O::sub(O::mul(e1[0], e2[1]), O::mul(e1[1], e2[0]));
  area = O::mul(R(0.5), O::sqrt_(O::add(O::add(O::mul(nx, nx), O::mul(ny, ny)), O::mul(nz, nz))));
}

template <typename R>
struct Axis {
  const R* faces;   // n+1 values (device)
  const R* widths;  // n values (device)
  R lo, hi, h;      // faces[0], faces[n], width when uniform
  R inv_h;          // 1/h when uniform (rounded)
  int n;
  int periodic;
  int uniform;
  // Non-uniform axes: [lo, hi) cut into nbk equal buckets; bucket[b] is the
  // cell containing the bucket's lower edge (device, nbk values).
  const int* bucket;
  R inv_bw;         // nbk / (hi - lo) (rounded)
  int nbk;
};

template <typename R>
struct Grid {
  Axis<R> ax[3];
};

// Spreading tiles: 2^l home cells per axis; bins = tiles + 1 (the last bin
// collects dropped markers).
struct Tiles {
  int l[3];
  int nb[3];
  int nbins;
};

// Home cell of coordinate x on one axis: face_i <= x < face_{i+1}.  Returns -1
// outside [faces[0], faces[n]) or for NaN.  Uniform axes guess i from
// (x - lo) * (1/h), other axes take the cell of x's bucket; the guess is then
// corrected against the face array, so the result agrees with the exact
// comparison whatever the rounding of the guess (a bucket holds only a few
// faces, so the corrections take few steps).
template <typename R>
__device__ __forceinline__ int locate_axis(const Axis<R>& a, R x) {
  if (!(x >= a.lo && x < a.hi)) return -1;
  int i;
  if (a.uniform) {
    R s = (x - a.lo) * a.inv_h;
    i = (int)s;
    i = i < 0 ? 0 : (i > a.n - 1 ? a.n - 1 : i);
    if (x < a.faces[i]) --i;
    else if (x >= a.faces[i + 1]) ++i;
  } else {
    int b = (int)((x - a.lo) * a.inv_bw);
    b = b < 0 ? 0 : (b > a.nbk - 1 ? a.nbk - 1 : b);
    i = __ldg(a.bucket + b);
    while (i > 0 && x < a.faces[i]) --i;
    while (i < a.n - 1 && x >= a.faces[i + 1]) ++i;
  }
  return i;
}

// A home index is usable when the 3-wide support stays on the grid (always on
// periodic axes, which wrap).
template <typename R>
__device__ __forceinline__ bool support_ok(const Axis<R>& a, int i) {
  return i >= 0 && (a.periodic || (i >= 1 && i <= a.n - 2));
}

__device__ __forceinline__ int wrap(int j, int n, int periodic) {
  if (periodic) return j < 0 ? j + n : (j >= n ? j - n : j);
  return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

template <typename R>
__device__ __forceinline__ R width_of(const Axis<R>& a, int j) {
  return a.uniform ? a.h : a.widths[j];
}

// Geometry of the 3 support nodes of one axis, in units of the home cell's
// width: xi[a] = (x_node - x_l)/Delta_home, node widths w[a] (physical), the
// marker's position frac in [0, 1) across the home cell and t = frac - 1/2,
// its offset from the home-cell centre.
template <typename R>
struct AxisNodes {
  R xi[3];
  R w[3];
  R frac;
  R t;
};

// On a uniform axis both width ratios are exactly 1 and the offset is
// (x - face_i) * (1/h), which equals (x - face_i)/h when h is a power of two.
template <typename R>
__device__ __forceinline__ AxisNodes<R> axis_nodes(const Axis<R>& a, int i, R x) {
  AxisNodes<R> s;
  if (a.uniform) {
    s.frac = (x - a.faces[i]) * a.inv_h;
    s.t = s.frac - R(0.5);
    s.xi[0] = R(-1) - s.t;
    s.xi[1] = -s.t;
    s.xi[2] = R(1) - s.t;
    s.w[0] = s.w[1] = s.w[2] = a.h;
    return s;
  }
  const R wh = width_of(a, i);
  const R wm = width_of(a, wrap(i - 1, a.n, a.periodic));
  const R wp = width_of(a, wrap(i + 1, a.n, a.periodic));
  s.frac = (x - a.faces[i]) / wh;
  s.t = s.frac - R(0.5);
  s.xi[0] = -(R(0.5) + R(0.5) * (wm / wh)) - s.t;
  s.xi[1] = -s.t;
  s.xi[2] = (R(0.5) + R(0.5) * (wp / wh)) - s.t;
  s.w[0] = wm;
  s.w[1] = wh;
  s.w[2] = wp;
  return s;
}

// Node geometry at a prescribed offset t with neighbour/home width ratios
// rm, rp (used to tabulate fast-MLS shape functions on the sub-Eulerian mesh).
template <typename R>
__device__ __forceinline__ AxisNodes<R> axis_nodes_at(R t, R wm, R wh, R wp) {
  AxisNodes<R> s;
  s.t = t;
  s.frac = t + R(0.5);
  s.xi[0] = -(R(0.5) + R(0.5) * (wm / wh)) - t;
  s.xi[1] = -t;
  s.xi[2] = (R(0.5) + R(0.5) * (wp / wh)) - t;
  s.w[0] = wm;
  s.w[1] = wh;
  s.w[2] = wp;
  return s;
}

template <typename R> __device__ __forceinline__ R dev_exp(R v);
// Single precision takes the hardware exponential: for the arguments here
// (|v| <= 4 with eps = 1) its relative error is a few ulp, far inside the
// single-precision tolerance of the shape functions.
template <> __device__ __forceinline__ float dev_exp<float>(float v) { return __expf(v); }

// 1/sqrt(d): the hardware reciprocal square root in single precision (about
// 1 ulp; the solve is followed by a refinement step), IEEE operations in double.
__device__ __forceinline__ float inv_sqrt(float d) { return rsqrtf(d); }
__device__ __forceinline__ double inv_sqrt(double d) { return 1.0 / sqrt(d); }
template <> __device__ __forceinline__ double dev_exp<double>(double v) { return exp(v); }

// 4x4 symmetric positive definite solve by Cholesky, A packed lower-triangular
// row by row: a00 a10 a11 a20 a21 a22 a30 a31 a32 a33.
template <typename R>
struct Chol4 {
  R l10, l20, l21, l30, l31, l32;
  R i0, i1, i2, i3;   // reciprocals of the diagonal of L
  bool ok;

  __device__ __forceinline__ void factor(const R a[10]) {
    R d0 = a[0];
    ok = d0 > R(0);
    i0 = inv_sqrt(d0);
    l10 = a[1] * i0;
    l20 = a[3] * i0;
    l30 = a[6] * i0;
    R d1 = a[2] - l10 * l10;
    ok = ok && d1 > R(0);
    i1 = inv_sqrt(d1);
    l21 = (a[4] - l20 * l10) * i1;
    l31 = (a[7] - l30 * l10) * i1;
    R d2 = a[5] - l20 * l20 - l21 * l21;
    ok = ok && d2 > R(0);
    i2 = inv_sqrt(d2);
    l32 = (a[8] - l30 * l20 - l31 * l21) * i2;
    R d3 = a[9] - l30 * l30 - l31 * l31 - l32 * l32;
    ok = ok && d3 > R(0);
    i3 = inv_sqrt(d3);
  }

  __device__ __forceinline__ void solve(const R b[4], R y[4]) const {
    R z0 = b[0] * i0;
    R z1 = (b[1] - l10 * z0) * i1;
    R z2 = (b[2] - l20 * z0 - l21 * z1) * i2;
    R z3 = (b[3] - l30 * z0 - l31 * z1 - l32 * z2) * i3;
    y[3] = z3 * i3;
    y[2] = (z2 - l32 * y[3]) * i2;
    y[1] = (z1 - l21 * y[2] - l31 * y[3]) * i1;
    y[0] = (z0 - l10 * y[1] - l20 * y[2] - l30 * y[3]) * i0;
  }
};

template <typename R>
__device__ __forceinline__ void sym_mul(const R a[10], const R y[4], R out[4]) {
  out[0] = a[0] * y[0] + a[1] * y[1] + a[3] * y[2] + a[6] * y[3];
  out[1] = a[1] * y[0] + a[2] * y[1] + a[4] * y[2] + a[7] * y[3];
  out[2] = a[3] * y[0] + a[4] * y[1] + a[5] * y[2] + a[8] * y[3];
  out[3] = a[6] * y[0] + a[7] * y[1] + a[8] * y[2] + a[9] * y[3];
}

// 1-norm condition number of the packed SPD matrix from its Cholesky factor:
// ||A||_1 ||A^-1||_1 with A^-1 = M^T M, M = L^-1 (lower triangular, formed
// column by column from L M = I).
template <typename R>
__device__ __forceinline__ R cond1(const R a[10], const Chol4<R>& ch) {
  R colsum[4] = {
      fabs(a[0]) + fabs(a[1]) + fabs(a[3]) + fabs(a[6]),
      fabs(a[1]) + fabs(a[2]) + fabs(a[4]) + fabs(a[7]),
      fabs(a[3]) + fabs(a[4]) + fabs(a[5]) + fabs(a[8]),
      fabs(a[6]) + fabs(a[7]) + fabs(a[8]) + fabs(a[9])};
  const R an = fmax(fmax(colsum[0], colsum[1]), fmax(colsum[2], colsum[3]));
  const R m00 = ch.i0, m11 = ch.i1, m22 = ch.i2, m33 = ch.i3;
  const R m10 = -ch.l10 * m00 * m11;
  const R m21 = -ch.l21 * m11 * m22;
  const R m20 = -(ch.l20 * m00 + ch.l21 * m10) * m22;
  const R m32 = -ch.l32 * m22 * m33;
  const R m31 = -(ch.l31 * m11 + ch.l32 * m21) * m33;
  const R m30 = -(ch.l30 * m00 + ch.l31 * m10 + ch.l32 * m20) * m33;
  const R b00 = m00 * m00 + m10 * m10 + m20 * m20 + m30 * m30;
  const R b01 = m10 * m11 + m20 * m21 + m30 * m31;
  const R b02 = m20 * m22 + m30 * m32;
  const R b03 = m30 * m33;
  const R b11 = m11 * m11 + m21 * m21 + m31 * m31;
  const R b12 = m21 * m22 + m31 * m32;
  const R b13 = m31 * m33;
  const R b22 = m22 * m22 + m32 * m32;
  const R b23 = m32 * m33;
  const R b33 = m33 * m33;
  const R inv_n = fmax(fmax(fabs(b00) + fabs(b01) + fabs(b02) + fabs(b03), fabs(b01) + fabs(b11) + fabs(b12) + fabs(b13)),
                       fmax(fabs(b02) + fabs(b12) + fabs(b22) + fabs(b23), fabs(b03) + fabs(b13) + fabs(b23) + fabs(b33)));
  return an * inv_n;
}

// Exact-MLS solve of one marker from its per-axis node geometry.
//   Eq. 3: A = sum_k W_k p_k p_k^T with p_k = [1, xi_x, xi_y, xi_z] (marker-
//          centred, home-width-scaled basis, an affine change of [1,x,y,z]
//          under which Phi is invariant), W_k = exp(-|xi_k|^2/eps^2)
//          evaluated as the product of three per-axis factors w[d][a].
//   Eq. 6: Phi^T = p^T(x_l) A^-1 B = e_0^T A^-1 B, i.e. phi_k = W_k (y . p_k)
//          with A y = e_0 (A is symmetric).
// `refine` extra residual-correction steps are applied to y.  Returns false
// if A is not numerically positive definite; `cond` (if non-null) receives
// cond_1(A).
template <typename R>
__device__ __forceinline__ bool exact_solve(const AxisNodes<R> s[3], R inv_eps2, int refine, R w[3][3], R y[4],
                                            R* cond) {
  // Per-axis weights and moments S_m[d] = sum_a w[d][a] xi[d][a]^m.  The
  // weight and the stencil are tensor products, so every entry of the
  // 27-term sum of Eq. 3 factorises into a product of three of them, e.g.
  // A_xy = sum_abc w_a w_b w_c xi_a xi_b = S1[x] S1[y] S0[z].
  R S0[3], S1[3], S2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    S0[d] = S1[d] = S2[d] = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const R xi = s[d].xi[a];
      const R wa = dev_exp<R>(-(xi * xi) * inv_eps2);
      w[d][a] = wa;
      S0[d] += wa;
      S1[d] += wa * xi;
      S2[d] += wa * xi * xi;
    }
  }
  R A[10];
  A[0] = S0[0] * S0[1] * S0[2];
  A[1] = S1[0] * S0[1] * S0[2];
  A[2] = S2[0] * S0[1] * S0[2];
  A[3] = S0[0] * S1[1] * S0[2];
  A[4] = S1[0] * S1[1] * S0[2];
  A[5] = S0[0] * S2[1] * S0[2];
  A[6] = S0[0] * S0[1] * S1[2];
  A[7] = S1[0] * S0[1] * S1[2];
  A[8] = S0[0] * S1[1] * S1[2];
  A[9] = S0[0] * S0[1] * S2[2];

  Chol4<R> ch;
  ch.factor(A);
  if (!ch.ok) return false;
  const R e0[4] = {R(1), R(0), R(0), R(0)};
  ch.solve(e0, y);
  for (int it = 0; it < refine; ++it) {
    R Ay[4], r[4], dy[4];
    sym_mul(A, y, Ay);
    r[0] = R(1) - Ay[0];
    r[1] = -Ay[1];
    r[2] = -Ay[2];
    r[3] = -Ay[3];
    ch.solve(r, dy);
    y[0] += dy[0];
    y[1] += dy[1];
    y[2] += dy[2];
    y[3] += dy[3];
  }
  if (cond) *cond = cond1(A, ch);
  return true;
}

// Streams phi_k = W_k (y . p_k) = wx_a wy_b wz_c (y0 + y1 xi_x,a + y2 xi_y,b +
// y3 xi_z,c) for k = 9c + 3b + a, with the (b, c) products formed once.
template <typename R, typename Sink>
__device__ __forceinline__ void exact_emit(const AxisNodes<R> s[3], const R w[3][3], const R y[4], Sink&& sink) {
  R gx[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) gx[a] = y[0] + y[1] * s[0].xi[a];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const R wyz = w[1][b] * w[2][c];
      const R gyz = y[2] * s[1].xi[b] + y[3] * s[2].xi[c];
#pragma unroll
      for (int a = 0; a < 3; ++a) sink(a, b, c, (w[0][a] * wyz) * (gx[a] + gyz));
    }
}

// c_l of Eq. 8 for an exact-MLS marker without forming the 27 terms: with
// phi_abc = X_a Y_b Z_c (y0 + y1 xi_x,a + y2 xi_y,b + y3 xi_z,c) (the Gaussian
// W = X Y Z is separable) and node widths Dx_a, Dy_b, Dz_c, the sums
// sum_k phi_k Dx_k, sum_k phi_k Dy_k, sum_k phi_k Dz_k and sum_k phi_k dV_k
// factorise into the per-axis sums S0 = sum_a W_a, S1 = sum_a W_a xi_a,
// Q0 = sum_a W_a D_a and Q1 = sum_a W_a xi_a D_a (the same sums, reassociated).
// Returns 0 when sum_k phi_k dV_k is 0.
template <typename R>
__device__ __forceinline__ R exact_scale(const AxisNodes<R> s[3], const R w[3][3], const R y[4], R area) {
  R S0[3], S1[3], Q0[3], Q1[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    S0[d] = S1[d] = Q0[d] = Q1[d] = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const R W = w[d][a], Wxi = W * s[d].xi[a];
      S0[d] += W;
      S1[d] += Wxi;
      Q0[d] += W * s[d].w[a];
      Q1[d] += Wxi * s[d].w[a];
    }
  }
  const R hx = S0[1] * S0[2] * (y[0] * Q0[0] + y[1] * Q1[0]) + (y[2] * S1[1] * S0[2] + y[3] * S0[1] * S1[2]) * Q0[0];
  const R hy = S0[0] * S0[2] * (y[0] * Q0[1] + y[2] * Q1[1]) + (y[1] * S1[0] * S0[2] + y[3] * S0[0] * S1[2]) * Q0[1];
  const R hz = S0[0] * S0[1] * (y[0] * Q0[2] + y[3] * Q1[2]) + (y[1] * S1[0] * S0[1] + y[2] * S0[0] * S1[1]) * Q0[2];
  const R vol = Q0[0] * Q0[1] * Q0[2] * y[0] + Q1[0] * Q0[1] * Q0[2] * y[1] + Q0[0] * Q1[1] * Q0[2] * y[2] +
                Q0[0] * Q0[1] * Q1[2] * y[3];
  return vol != R(0) ? (area * ((hx + hy + hz) / R(3))) / vol : R(0);
}

// ---- quadratic basis (m = 10) ------------------------------------------------
// Section 2 takes the basis from Pascal's pyramid and leaves m free; the
// quadratic option is p = [1, xi_x, xi_y, xi_z, xi_x^2, xi_y^2, xi_z^2,
// xi_x xi_y, xi_y xi_z, xi_z xi_x] in the same marker-centred, home-width-scaled
// coordinates (an affine change that maps the quadratic space onto itself, so
// Phi is unchanged and p(x_l) = e_0).  quad_exp(i, d) is the exponent of axis d
// in term i; with the tensor-product weight every entry of A is a product of
// three per-axis moments, A_ij = prod_d S_{e_i,d + e_j,d}[d], S_m = sum_a w_a xi_a^m.
constexpr int kQuad = 10;
constexpr int kQuadPacked = kQuad * (kQuad + 1) / 2;

__host__ __device__ constexpr int quad_exp(int i, int d) {
  return i == 0   ? 0
         : i <= 3 ? (i - 1 == d ? 1 : 0)
         : i <= 6 ? (i - 4 == d ? 2 : 0)
         : i == 7 ? (d == 0 || d == 1 ? 1 : 0)
         : i == 8 ? (d == 1 || d == 2 ? 1 : 0)
                  : (d == 2 || d == 0 ? 1 : 0);
}

__host__ __device__ constexpr int packed(int i, int j) { return i * (i + 1) / 2 + j; }  // i >= j

template <typename R>
__device__ __forceinline__ R quad_entry(const R S[3][5], int i, int j) {
  return S[0][quad_exp(i, 0) + quad_exp(j, 0)] * S[1][quad_exp(i, 1) + quad_exp(j, 1)] *
         S[2][quad_exp(i, 2) + quad_exp(j, 2)];
}

// In-place Cholesky of the packed lower triangle (row by row, i >= j); the
// diagonal slots end up holding 1/L_ii.  Returns false unless every pivot is
// positive.
template <typename R>
__device__ __forceinline__ bool quad_factor(R L[kQuadPacked]) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < kQuad; ++j) {
    R d = L[packed(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= L[packed(j, k)] * L[packed(j, k)];
    ok = ok && d > R(0);
    const R inv = inv_sqrt(d);
    L[packed(j, j)] = inv;
#pragma unroll
    for (int i = j + 1; i < kQuad; ++i) {
      R v = L[packed(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= L[packed(i, k)] * L[packed(j, k)];
      L[packed(i, j)] = v * inv;
    }
  }
  return ok;
}

template <typename R>
__device__ __forceinline__ void quad_solve(const R L[kQuadPacked], const R b[kQuad], R y[kQuad]) {
  R z[kQuad];
#pragma unroll
  for (int i = 0; i < kQuad; ++i) {
    R v = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) v -= L[packed(i, k)] * z[k];
    z[i] = v * L[packed(i, i)];
  }
#pragma unroll
  for (int i = kQuad - 1; i >= 0; --i) {
    R v = z[i];
#pragma unroll
    for (int k = i + 1; k < kQuad; ++k) v -= L[packed(k, i)] * y[k];
    y[i] = v * L[packed(i, i)];
  }
}

// Exact-MLS solve with the quadratic basis: as exact_solve, A y = e_0 with
// `refine` residual corrections (A re-formed from the moments), cond_1(A)
// from the column sums of A and of A^-1 = M^T M, M = L^-1 (lower triangular,
// row by row from L M = I), as for the linear basis.
template <typename R>
__device__ __forceinline__ bool exact_solve_quad(const AxisNodes<R> s[3], R inv_eps2, int refine, R w[3][3],
                                                 R y[kQuad], R* cond) {
  R S[3][5];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int m = 0; m < 5; ++m) S[d][m] = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const R xi = s[d].xi[a];
      const R wa = dev_exp<R>(-(xi * xi) * inv_eps2);
      w[d][a] = wa;
      R pw = wa;
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        S[d][m] += pw;
        pw *= xi;
      }
    }
  }
  R L[kQuadPacked];
#pragma unroll
  for (int i = 0; i < kQuad; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) L[packed(i, j)] = quad_entry(S, i, j);
  if (!quad_factor(L)) return false;
  R e0[kQuad];
#pragma unroll
  for (int i = 0; i < kQuad; ++i) e0[i] = i == 0 ? R(1) : R(0);
  quad_solve(L, e0, y);
  for (int it = 0; it < refine; ++it) {
    R r[kQuad], dy[kQuad];
#pragma unroll
    for (int i = 0; i < kQuad; ++i) {
      R v = e0[i];
#pragma unroll
      for (int j = 0; j < kQuad; ++j) v -= quad_entry(S, i, j) * y[j];
      r[i] = v;
    }
    quad_solve(L, r, dy);
#pragma unroll
    for (int i = 0; i < kQuad; ++i) y[i] += dy[i];
  }
  if (cond) {
    R Mi[kQuadPacked];
#pragma unroll
    for (int i = 0; i < kQuad; ++i) {
      Mi[packed(i, i)] = L[packed(i, i)];
#pragma unroll
      for (int j = 0; j < i; ++j) {
        R v = R(0);
#pragma unroll
        for (int k = j; k < i; ++k) v += L[packed(i, k)] * Mi[packed(k, j)];
        Mi[packed(i, j)] = -v * L[packed(i, i)];
      }
    }
    R col[kQuad], icol[kQuad];
#pragma unroll
    for (int i = 0; i < kQuad; ++i) col[i] = icol[i] = R(0);
#pragma unroll
    for (int i = 0; i < kQuad; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) {
        const R a = fabs(quad_entry(S, i, j));
        R b = R(0);
#pragma unroll
        for (int k = i; k < kQuad; ++k) b += Mi[packed(k, i)] * Mi[packed(k, j)];
        b = fabs(b);
        col[j] += a;
        icol[j] += b;
        if (i != j) {
          col[i] += a;
          icol[i] += b;
        }
      }
    R an = R(0), inv_n = R(0);
#pragma unroll
    for (int i = 0; i < kQuad; ++i) {
      an = fmax(an, col[i]);
      inv_n = fmax(inv_n, icol[i]);
    }
    *cond = an * inv_n;
  }
  return true;
}

// phi_k = W_k (y . p_k) for the quadratic basis, k = 9c + 3b + a: the terms
// without xi_x are formed once per (b, c), the rest as xi_x (g1 + y4 xi_x).
template <typename R, typename Sink>
__device__ __forceinline__ void exact_emit_quad(const AxisNodes<R> s[3], const R w[3][3], const R y[kQuad],
                                                Sink&& sink) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const R wyz = w[1][b] * w[2][c];
      const R yb = s[1].xi[b], zc = s[2].xi[c];
      const R g0 = y[0] + y[2] * yb + y[3] * zc + y[5] * (yb * yb) + y[6] * (zc * zc) + y[8] * (yb * zc);
      const R g1 = y[1] + y[7] * yb + y[9] * zc;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R xa = s[0].xi[a];
        sink(a, b, c, (w[0][a] * wyz) * (g0 + xa * (g1 + y[4] * xa)));
      }
    }
}

// Basis-size dispatch: MB = 4 (linear) or kQuad (quadratic).
template <int MB, typename R>
__device__ __forceinline__ bool exact_solve_m(const AxisNodes<R> s[3], R inv_eps2, int refine, R w[3][3], R y[MB],
                                              R* cond) {
  if constexpr (MB == 4)
    return exact_solve(s, inv_eps2, refine, w, y, cond);
  else
    return exact_solve_quad(s, inv_eps2, refine, w, y, cond);
}

template <int MB, typename R, typename Sink>
__device__ __forceinline__ void exact_emit_m(const AxisNodes<R> s[3], const R w[3][3], const R y[MB], Sink&& sink) {
  if constexpr (MB == 4)
    exact_emit(s, w, y, sink);
  else
    exact_emit_quad(s, w, y, sink);
}

// All 27 exact shape functions (table path).
template <typename R, int MB = 4>
__device__ __forceinline__ bool shape_exact(const AxisNodes<R> s[3], R inv_eps2, int refine, R phi[27],
                                            R* cond) {
  R w[3][3], y[MB];
  if (!exact_solve_m<MB>(s, inv_eps2, refine, w, y, cond)) return false;
  exact_emit_m<MB>(s, w, y, [&](int a, int b, int c, R v) { phi[9 * c + 3 * b + a] = v; });
  return true;
}

// Running sums for c_l of Eq. 8 while phi is streamed out.
template <typename R>
struct ScaleSums {
  R mx[3], my[3], mz[3], vol;
  __device__ __forceinline__ ScaleSums() {
#pragma unroll
    for (int q = 0; q < 3; ++q) mx[q] = my[q] = mz[q] = R(0);
    vol = R(0);
  }
  __device__ __forceinline__ void add(const AxisNodes<R> s[3], int a, int b, int c, R p) {
    mx[a] += p;
    my[b] += p;
    mz[c] += p;
    vol += p * (s[0].w[a] * s[1].w[b] * s[2].w[c]);
  }
  // c_l = A_l h_l / sum_k phi_k dV_k, h_l = sum_k phi_k (Dx_k + Dy_k + Dz_k)/3.
  __device__ __forceinline__ R scale(const AxisNodes<R> s[3], R area) const {
    R hsum = R(0);
#pragma unroll
    for (int q = 0; q < 3; ++q) hsum += mx[q] * s[0].w[q] + my[q] * s[1].w[q] + mz[q] * s[2].w[q];
    return (area * (hsum / R(3))) / vol;
  }
};

}  // namespace mls
