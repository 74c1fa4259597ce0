// Device-side pieces shared by the kernels that build transfer functions:
// the build arguments, the per-marker prologue (home cell and support
// geometry) and epilogue, and the field access of an interpolation fused into
// a build.
#pragma once

#include <cmath>
#include <limits>

#include "mls_host.h"

namespace mls {

template <typename R>
struct BuildArgs {
  Grid<R> g;
  Grid<double> gd;       // double-precision grid for the conditioning fallback
  const R* x;
  const R* area;
  const int32_t* perm;
  int64_t M, cap;
  R* phi;
  R* c;
  int32_t* home;
  unsigned long long* status;
  int32_t* redo;         // markers whose single-precision solve is redone in double (count in status[2])
  R inv_eps2;
  double inv_eps2_d;
  int refine;
  int want_cond;         // single precision with cond_max > 0
  float cond_max_f;      // cond_max rounded down to float: cond > cond_max_f <=> cond > cond_max
  // fast-MLS
  const R* table;
  int class_axis;
  int n_sub;
};

// Shared prologue: fetch marker perm[j], locate its home cell, and build the
// per-axis node geometry.  Dropped markers get phi = 0, c = 0, home = -1.
template <typename R>
__device__ __forceinline__ bool marker_setup(const BuildArgs<R>& a, int64_t j, int h[3], R p[3],
                                             AxisNodes<R> s[3], R& ar) {
  const int64_t m = a.perm[j];
  p[0] = a.x[m];
  p[1] = a.x[a.M + m];
  p[2] = a.x[2 * a.M + m];
  ar = a.area[m];
  bool ok = isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]) && isfinite(ar);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    h[d] = locate_axis(a.g.ax[d], p[d]);
    ok = ok && support_ok(a.g.ax[d], h[d]);
  }
  if (!ok) {
#pragma unroll
    for (int k = 0; k < 27; ++k) a.phi[k * a.cap + j] = R(0);
    a.c[j] = R(0);
    a.home[j] = -1;
    return false;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) s[d] = axis_nodes(a.g.ax[d], h[d], p[d]);
  return true;
}

template <typename R>
__device__ __forceinline__ void marker_finish(const BuildArgs<R>& a, int64_t j, const int h[3],
                                              const AxisNodes<R> s[3], const ScaleSums<R>& sums, R ar) {
  a.c[j] = sums.vol != R(0) ? sums.scale(s, ar) : R(0);
  a.home[j] = (h[2] * a.g.ax[1].n + h[1]) * a.g.ax[0].n + h[0];
}

// The field and output of an interpolation fused into the exact build:
// u[3][N] (float, bfloat16 or double storage), U[3][M] in the real type.
template <typename R, typename FT>
struct InterpOut {
  const FT* u;
  R* U;            // or nullptr: U is formed but not stored
  int64_t N;
  // Direct forcing (optional, F != nullptr): F_l = (V_b,l - U_l) / dt.
  const R* Vb;
  R inv_dt;
  R* F;
  // U (and F) of marker m in the caller's order; dropped markers get zeros.
  __device__ __forceinline__ void store(int64_t m, int64_t M, R U0, R U1, R U2) const {
    if (U) {
      U[m] = U0;
      U[M + m] = U1;
      U[2 * M + m] = U2;
    }
    if (F) {
      F[m] = (Vb[m] - U0) * inv_dt;
      F[M + m] = (Vb[M + m] - U1) * inv_dt;
      F[2 * M + m] = (Vb[2 * M + m] - U2) * inv_dt;
    }
  }
  __device__ __forceinline__ void store_zero(int64_t m, int64_t M) const {
    if (U) U[m] = U[M + m] = U[2 * M + m] = R(0);
    if (F) F[m] = F[M + m] = F[2 * M + m] = R(0);
  }
};

template <typename R, typename FT> __device__ __forceinline__ R field_value(const FT* p);
template <> __device__ __forceinline__ float field_value<float, float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float field_value<float, __nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ double field_value<double, double>(const double* p) { return __ldg(p); }

// Offsets inside one field component (n_x n_y n_z < 2^31) of the 27 support
// nodes of home cell h: x index per a, row offset (z, y) per (c, b).
template <typename R>
__device__ __forceinline__ void support_offsets(const Grid<R>& g, const int h[3], int xs[3], int rows[3][3]) {
  int ys[3], zs[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    xs[q] = wrap(h[0] + q - 1, g.ax[0].n, g.ax[0].periodic);
    ys[q] = wrap(h[1] + q - 1, g.ax[1].n, g.ax[1].periodic);
    zs[q] = wrap(h[2] + q - 1, g.ax[2].n, g.ax[2].periodic);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b) rows[c][b] = (zs[c] * g.ax[1].n + ys[b]) * g.ax[0].n;
}

// Build arguments of a context and transfer (host).
template <typename R>
inline BuildArgs<R> make_args(const mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M) {
  BuildArgs<R> a;
  a.g = device_grid<R>(ctx);
  a.gd = device_grid<double>(ctx);
  a.x = (const R*)x;
  a.area = (const R*)area;
  a.perm = T->perm;
  a.M = M;
  a.cap = T->cap;
  a.phi = (R*)T->phi;
  a.c = (R*)T->c;
  a.home = T->home;
  a.status = T->status;
  a.redo = T->key;  // free once the tile sort has scattered
  a.inv_eps2 = (R)(1.0 / (ctx->opt.eps * ctx->opt.eps));
  a.inv_eps2_d = 1.0 / (ctx->opt.eps * ctx->opt.eps);
  a.refine = ctx->opt.real == MLS_F32 ? ctx->opt.refine : 0;
  a.want_cond = ctx->opt.real == MLS_F32 && ctx->opt.cond_max > 0.0;
  float t = (float)ctx->opt.cond_max;
  if ((double)t > ctx->opt.cond_max) t = std::nextafter(t, -std::numeric_limits<float>::infinity());
  a.cond_max_f = t;
  a.table = (const R*)ctx->table;
  a.class_axis = ctx->class_axis;
  a.n_sub = ctx->opt.n_sub;
  return a;
}

}  // namespace mls
