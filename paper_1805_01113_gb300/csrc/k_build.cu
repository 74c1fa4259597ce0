// Shape-function builds: exact-MLS (Eqs. 3-6), the fast-MLS table of exact
// shape functions on the sub-Eulerian mesh, and fast-MLS (Eqs. 9-10).
// One thread per marker, markers visited in tile order (perm), so phi[k][j],
// c[j] and home[j] are written with unit stride across a warp.
#include <algorithm>
#include <cmath>
#include <limits>

#include "build_common.cuh"

namespace mls {

template <typename R> struct TableVec;
template <> struct TableVec<float> { using type = float4; };
template <> struct TableVec<double> { using type = double2; };

// Exact-MLS build (Eqs. 3-6, 8): phi is written node by node as it is formed.
// A single-precision solve that is ill-conditioned (cond_1(A) > cond_max) or
// not numerically SPD queues the marker for k_build_exact_redo instead.
// MB is the basis size: 4 (linear, the paper's) or kQuad (quadratic).
template <typename R, int MB>
__global__ void __launch_bounds__(kBlock, MB == 4 && sizeof(R) == 4 ? 4 : 1) k_build_exact(BuildArgs<R> a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.M) return;
  int h[3];
  R p[3], ar;
  AxisNodes<R> s[3];
  if (!marker_setup(a, j, h, p, s, ar)) return;
  R w[3][3], y[MB];
  R cond = R(0);
  const bool want_cond = sizeof(R) == 4 && a.want_cond;
  bool good = exact_solve_m<MB>(s, a.inv_eps2, a.refine, w, y, want_cond ? &cond : nullptr);
  if (sizeof(R) == 4 && (!good || (want_cond && (float)cond > a.cond_max_f))) {
    a.redo[atomicAdd(&a.status[2], 1ULL)] = (int32_t)j;
    return;
  }
  R c = R(0);
  if (good) {
    if constexpr (MB == 4) {
      c = exact_scale(s, w, y, ar);
      exact_emit(s, w, y, [&](int q, int b, int cc, R v) { a.phi[(9 * cc + 3 * b + q) * a.cap + j] = v; });
    } else {
      ScaleSums<R> sums;
      exact_emit_m<MB>(s, w, y, [&](int q, int b, int cc, R v) {
        a.phi[(9 * cc + 3 * b + q) * a.cap + j] = v;
        sums.add(s, q, b, cc, v);
      });
      c = sums.vol != R(0) ? sums.scale(s, ar) : R(0);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 27; ++k) a.phi[k * a.cap + j] = R(0);
  }
  a.c[j] = c;
  a.home[j] = (h[2] * a.g.ax[1].n + h[1]) * a.g.ax[0].n + h[0];
}

// The queued single-precision markers, solved in double and rounded
// (grid-stride over the queue that k_build_exact filled).
template <int MB>
__global__ void __launch_bounds__(kBlock) k_build_exact_redo(BuildArgs<float> a) {
  const unsigned long long n = a.status[2];
  for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (unsigned long long)gridDim.x * blockDim.x) {
    const int64_t j = a.redo[q];
    int h[3];
    float p[3], ar;
    AxisNodes<float> s[3];
    if (!marker_setup(a, j, h, p, s, ar)) continue;
    AxisNodes<double> sd[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) sd[d] = axis_nodes(a.gd.ax[d], h[d], (double)p[d]);
    double wd[3][3], yd[MB];
    const bool good = exact_solve_m<MB>(sd, a.inv_eps2_d, 0, wd, yd, (double*)nullptr);
    ScaleSums<float> sums;
    if (good) {
      exact_emit_m<MB>(sd, wd, yd, [&](int qq, int b, int c, double v) {
        a.phi[(9 * c + 3 * b + qq) * a.cap + j] = (float)v;
        sums.add(s, qq, b, c, (float)v);
      });
    } else {
#pragma unroll
      for (int k = 0; k < 27; ++k) a.phi[k * a.cap + j] = 0.f;
    }
    marker_finish(a, j, h, s, sums, ar);
  }
}

// Exact-MLS build (Eqs. 3-6, 8) with the interpolation U_l = sum_k phi_k u_k
// (text after Eq. 6) of the same markers: each phi_k is stored, as in
// k_build_exact, and multiplied into the three sums with the field at its
// node as it is formed, so the interpolation reads no phi.  Markers queued for the double re-solve
// get U from k_build_exact_interp_redo; dropped markers get U = 0.
// Held to 64 registers (four blocks per SM, as k_build_exact): the field loads
// of more resident warps overlap (1.97 ms on 32 M markers, against 2.17 ms at
// 80 registers and 2.07 ms at 48 registers with spills).
template <typename R, typename FT>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 4 : 1) k_build_exact_interp(BuildArgs<R> a,
                                                                                      InterpOut<R, FT> io) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.M) return;
  int h[3];
  R p[3], ar;
  AxisNodes<R> s[3];
  const int64_t m = a.perm[j];
  if (!marker_setup(a, j, h, p, s, ar)) {
    io.store_zero(m, a.M);
    return;
  }
  R w[3][3], y[4];
  R cond = R(0);
  const bool want_cond = sizeof(R) == 4 && a.want_cond;
  const bool good = exact_solve_m<4>(s, a.inv_eps2, a.refine, w, y, want_cond ? &cond : nullptr);
  if (sizeof(R) == 4 && (!good || (want_cond && (float)cond > a.cond_max_f))) {
    a.redo[atomicAdd(&a.status[2], 1ULL)] = (int32_t)j;
    return;
  }
  R U0 = R(0), U1 = R(0), U2 = R(0), c = R(0);
  if (good) {
    int xs[3];
    int rows[3][3];
    support_offsets(a.g, h, xs, rows);
    const FT* u0 = io.u;
    const FT* u1 = u0 + io.N;
    const FT* u2 = u1 + io.N;
    c = exact_scale(s, w, y, ar);
    exact_emit(s, w, y, [&](int q, int b, int cc, R v) {
      a.phi[(9 * cc + 3 * b + q) * a.cap + j] = v;
      const int o = rows[cc][b] + xs[q];
      U0 += v * field_value<R, FT>(u0 + o);
      U1 += v * field_value<R, FT>(u1 + o);
      U2 += v * field_value<R, FT>(u2 + o);
    });
  } else {
#pragma unroll
    for (int k = 0; k < 27; ++k) a.phi[k * a.cap + j] = R(0);
  }
  a.c[j] = c;
  a.home[j] = (h[2] * a.g.ax[1].n + h[1]) * a.g.ax[0].n + h[0];
  io.store(m, a.M, U0, U1, U2);
}

// The queued single-precision markers of k_build_exact_interp: solved in
// double and rounded as in k_build_exact_redo, then interpolated with the
// rounded phi.
template <typename FT>
__global__ void __launch_bounds__(kBlock) k_build_exact_interp_redo(BuildArgs<float> a, InterpOut<float, FT> io) {
  const unsigned long long n = a.status[2];
  for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (unsigned long long)gridDim.x * blockDim.x) {
    const int64_t j = a.redo[q];
    const int64_t m = a.perm[j];
    int h[3];
    float p[3], ar;
    AxisNodes<float> s[3];
    if (!marker_setup(a, j, h, p, s, ar)) {
      io.store_zero(m, a.M);
      continue;
    }
    AxisNodes<double> sd[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) sd[d] = axis_nodes(a.gd.ax[d], h[d], (double)p[d]);
    double wd[3][3], yd[4];
    const bool good = exact_solve_m<4>(sd, a.inv_eps2_d, 0, wd, yd, (double*)nullptr);
    ScaleSums<float> sums;
    float U0 = 0.f, U1 = 0.f, U2 = 0.f;
    if (good) {
      int xs[3];
      int rows[3][3];
      support_offsets(a.g, h, xs, rows);
      exact_emit_m<4>(sd, wd, yd, [&](int qq, int b, int c, double v) {
        const float f = (float)v;
        a.phi[(9 * c + 3 * b + qq) * a.cap + j] = f;
        sums.add(s, qq, b, c, f);
        const int o = rows[c][b] + xs[qq];
        U0 += f * field_value<float, FT>(io.u + o);
        U1 += f * field_value<float, FT>(io.u + io.N + o);
        U2 += f * field_value<float, FT>(io.u + 2 * io.N + o);
      });
    } else {
#pragma unroll
      for (int k = 0; k < 27; ++k) a.phi[k * a.cap + j] = 0.f;
    }
    marker_finish(a, j, h, s, sums, ar);
    io.store(m, a.M, U0, U1, U2);
  }
}

// Fast-MLS: the marker's position in its home cell picks the enclosing
// sub-cell of the n^3 sub-Eulerian mesh; the shape function is the Shepard
// blend of the 8 corner rows of the table, alpha_i proportional to 1/d_i^2
// (Eq. 10), evaluated as alpha_i = prod_{j!=i} d_j^2 / sum_i prod_{j!=i} d_j^2
// which equals it and stays finite when the marker sits on a corner.
template <typename R, bool SMEM>
__device__ __forceinline__ void fast_marker(const BuildArgs<R>& a, int64_t j, const R* __restrict__ table) {
  int h[3];
  R p[3], ar;
  AxisNodes<R> s[3];
  if (!marker_setup(a, j, h, p, s, ar)) return;
  const int n = a.n_sub, nm1 = n - 1;
  int sc[3];
  R lam[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const R u = s[d].frac * R(nm1);
    int q = (int)floor(u);
    q = q < 0 ? 0 : (q > nm1 - 1 ? nm1 - 1 : q);
    sc[d] = q;
    lam[d] = u - R(q);
  }
  R d2[8];
#pragma unroll
  for (int cidx = 0; cidx < 8; ++cidx) {
    const R dx = lam[0] - R(cidx & 1), dy = lam[1] - R((cidx >> 1) & 1), dz = lam[2] - R(cidx >> 2);
    d2[cidx] = dx * dx + dy * dy + dz * dz;
  }
  R pre[8], suf[8];
  pre[0] = R(1);
#pragma unroll
  for (int q = 1; q < 8; ++q) pre[q] = pre[q - 1] * d2[q - 1];
  suf[7] = R(1);
#pragma unroll
  for (int q = 6; q >= 0; --q) suf[q] = suf[q + 1] * d2[q + 1];
  R alpha[8], sum = R(0);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    alpha[q] = pre[q] * suf[q];
    sum += alpha[q];
  }
  const R inv = R(1) / sum;
  const int cl = a.class_axis >= 0 ? h[a.class_axis] : 0;
  const R* T = table + ((int64_t)cl * n * n * n + (int64_t)(((sc[2] * n) + sc[1]) * n + sc[0])) * kTableRow;
  // Corner q sits at sub-node offset (q&1, (q>>1)&1, q>>2) from the sub-cell origin.
  int roff[8];   // within one class's table: n^3 kTableRow values, far below 2^31
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    alpha[q] *= inv;
    roff[q] = ((((q >> 2) * n) + ((q >> 1) & 1)) * n + (q & 1)) * kTableRow;
  }
  // Rows are kTableRow = 28 values (27 + one pad), 16-byte aligned: read in
  // 16-byte vectors, kTableRow / kVec of them per corner.
  using V = typename TableVec<R>::type;
  constexpr int kVec = 16 / sizeof(R);
  ScaleSums<R> sums;
#pragma unroll
  for (int v = 0; v < kTableRow / kVec; ++v) {
    R acc[kVec];
#pragma unroll
    for (int e = 0; e < kVec; ++e) acc[e] = R(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const V* tp = reinterpret_cast<const V*>(T + roff[q]) + v;
      const V t = SMEM ? *tp : __ldg(tp);
      const R* tv = reinterpret_cast<const R*>(&t);
#pragma unroll
      for (int e = 0; e < kVec; ++e) acc[e] += alpha[q] * tv[e];
    }
#pragma unroll
    for (int e = 0; e < kVec; ++e) {
      const int k = v * kVec + e;
      if (k < 27) {
        a.phi[k * a.cap + j] = acc[e];
        sums.add(s, k % 3, (k / 3) % 3, k / 9, acc[e]);
      }
    }
  }
  marker_finish(a, j, h, s, sums, ar);
}

// Fast-MLS build (Eqs. 9-10), one thread per marker, table rows read through
// the read-only cache.
template <typename R>
__global__ void __launch_bounds__(kBlock) k_build_fast(BuildArgs<R> a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.M) return;
  fast_marker<R, false>(a, j, a.table);
}

// The same for a table that fits in shared memory (one class: grids uniform
// in all three axes): persistent blocks copy it once and read the 8 corner
// rows of every marker from shared memory instead of scattered cache lines.
// Blocks are larger than kBlock so that the two that fit per SM beside their
// table copies keep enough warps resident (two blocks of 512 at 64 registers).
constexpr int kFastSmemThreads = 512;
__global__ void __launch_bounds__(kFastSmemThreads, 2) k_build_fast_smem(BuildArgs<float> a, int table_vec4) {
  extern __shared__ float4 tab_s[];
  const float4* src = reinterpret_cast<const float4*>(a.table);
  for (int q = threadIdx.x; q < table_vec4; q += blockDim.x) tab_s[q] = src[q];
  __syncthreads();
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.M; j += (int64_t)gridDim.x * blockDim.x)
    fast_marker<float, true>(a, j, reinterpret_cast<const float*>(tab_s));
}

// Table of exact shape functions at the sub-Eulerian nodes -1/2 + i/(n-1)
// (faces included) of one home cell per class, computed in double and
// rounded to R.  A class is the home index along the single non-uniform axis;
// uniform axes have unit neighbour/home width ratios.
template <typename R, int MB>
__global__ void k_fast_table(Grid<double> gd, int class_axis, int64_t n_classes, int n_sub, double inv_eps2,
                             R* __restrict__ table) {
  const int64_t S3 = (int64_t)n_sub * n_sub * n_sub;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_classes * S3) return;
  const int64_t cl = idx / S3;
  const int s = (int)(idx % S3);
  const int sub[3] = {s % n_sub, (s / n_sub) % n_sub, s / (n_sub * n_sub)};
  AxisNodes<double> nd[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double t = -0.5 + (double)sub[d] / (double)(n_sub - 1);
    const Axis<double>& ax = gd.ax[d];
    if (d == class_axis) {
      const int i = (int)cl;
      nd[d] = axis_nodes_at(t, width_of(ax, wrap(i - 1, ax.n, ax.periodic)), width_of(ax, i),
                            width_of(ax, wrap(i + 1, ax.n, ax.periodic)));
    } else {
      const double w = width_of(ax, 0);
      nd[d] = axis_nodes_at(t, w, w, w);
    }
  }
  double phi[27];
  if (!shape_exact<double, MB>(nd, inv_eps2, 0, phi, nullptr)) {
    for (int k = 0; k < 27; ++k) phi[k] = 0.0;
  }
  for (int k = 0; k < 27; ++k) table[idx * kTableRow + k] = (R)phi[k];
  for (int k = 27; k < kTableRow; ++k) table[idx * kTableRow + k] = R(0);
}

template <int MB>
static void launch_build_exact_m(const mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M,
                                 cudaStream_t s) {
  const unsigned grid = (unsigned)((M + kBlock - 1) / kBlock);
  if (ctx->opt.real == MLS_F64)
    k_build_exact<double, MB><<<(unsigned)((M + kBlockF64 - 1) / kBlockF64), kBlockF64, 0, s>>>(
        make_args<double>(ctx, T, x, area, M));
  else {
    const BuildArgs<float> a = make_args<float>(ctx, T, x, area, M);
    k_build_exact<float, MB><<<grid, kBlock, 0, s>>>(a);
    const unsigned redo_grid = (unsigned)std::min<int64_t>(grid, 4 * 152);
    k_build_exact_redo<MB><<<redo_grid, kBlock, 0, s>>>(a);
  }
}

cudaError_t launch_build_exact(const mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M,
                               cudaStream_t s) {
  if (ctx->opt.basis == kQuad)
    launch_build_exact_m<kQuad>(ctx, T, x, area, M, s);
  else
    launch_build_exact_m<4>(ctx, T, x, area, M, s);
  return cudaGetLastError();
}

cudaError_t launch_build_exact_interp(const mls_ctx* ctx, mls_transfer* T, const void* x, const void* area,
                                      int64_t M, const void* u, void* U, cudaStream_t s, const void* Vb, double dt,
                                      void* F) {
  const int64_t N = (int64_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
  const double inv_dt = F ? 1.0 / dt : 0.0;
  if (ctx->opt.real == MLS_F64) {
    const InterpOut<double, double> io{(const double*)u, (double*)U, N, (const double*)Vb, inv_dt, (double*)F};
    k_build_exact_interp<double, double><<<(unsigned)((M + kBlockF64 - 1) / kBlockF64), kBlockF64, 0, s>>>(
        make_args<double>(ctx, T, x, area, M), io);
    return cudaGetLastError();
  }
  const unsigned grid = (unsigned)((M + kBlock - 1) / kBlock);
  const unsigned redo_grid = (unsigned)std::min<int64_t>(grid, 4 * 152);
  const BuildArgs<float> a = make_args<float>(ctx, T, x, area, M);
  if (ctx->opt.field == MLS_BF16) {
    const InterpOut<float, __nv_bfloat16> io{(const __nv_bfloat16*)u, (float*)U, N, (const float*)Vb, (float)inv_dt,
                                             (float*)F};
    k_build_exact_interp<float, __nv_bfloat16><<<grid, kBlock, 0, s>>>(a, io);
    k_build_exact_interp_redo<__nv_bfloat16><<<redo_grid, kBlock, 0, s>>>(a, io);
  } else {
    const InterpOut<float, float> io{(const float*)u, (float*)U, N, (const float*)Vb, (float)inv_dt, (float*)F};
    k_build_exact_interp<float, float><<<grid, kBlock, 0, s>>>(a, io);
    k_build_exact_interp_redo<float><<<redo_grid, kBlock, 0, s>>>(a, io);
  }
  return cudaGetLastError();
}

cudaError_t launch_build_fast(const mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M,
                              cudaStream_t s) {
  const unsigned grid = (unsigned)((M + kBlock - 1) / kBlock);
  if (ctx->opt.real == MLS_F64)
    k_build_fast<double><<<(unsigned)((M + kBlockF64 - 1) / kBlockF64), kBlockF64, 0, s>>>(
        make_args<double>(ctx, T, x, area, M));
  else if (ctx->fast_smem_grid > 0 && ctx->n_classes == 1) {
    const int64_t S3 = (int64_t)ctx->opt.n_sub * ctx->opt.n_sub * ctx->opt.n_sub;
    const int vec4 = (int)(S3 * kTableRow / 4);
    const unsigned g =
        (unsigned)std::min<int64_t>(ctx->fast_smem_grid, (M + kFastSmemThreads - 1) / kFastSmemThreads);
    k_build_fast_smem<<<g, kFastSmemThreads, (size_t)vec4 * 16, s>>>(make_args<float>(ctx, T, x, area, M), vec4);
  } else
    k_build_fast<float><<<grid, kBlock, 0, s>>>(make_args<float>(ctx, T, x, area, M));
  return cudaGetLastError();
}

// The shared-memory fast build is used when the single-precision table has
// one class and leaves room for two blocks per SM; its persistent grid is the
// resident block count.
cudaError_t build_configure(mls_ctx* ctx) {
  ctx->fast_smem_grid = 0;
  if (ctx->opt.real != MLS_F32 || !(ctx->uniform[0] && ctx->uniform[1] && ctx->uniform[2])) return cudaSuccess;
  const int64_t S3 = (int64_t)ctx->opt.n_sub * ctx->opt.n_sub * ctx->opt.n_sub;
  const int64_t bytes = S3 * kTableRow * 4;
  constexpr int kMaxTableBytes = 100 * 1024;
  if (bytes > kMaxTableBytes) return cudaSuccess;
  cudaError_t e = raise_smem_limit((const void*)k_build_fast_smem, (int)bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0, dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_fast_smem, kFastSmemThreads,
                                                     (size_t)bytes)) !=
      cudaSuccess)
    return e;
  ctx->fast_smem_grid = per_sm > 0 ? per_sm * sms : 0;
  return cudaSuccess;
}

cudaError_t launch_fast_table(mls_ctx* ctx, cudaStream_t s) {
  const int64_t S3 = (int64_t)ctx->opt.n_sub * ctx->opt.n_sub * ctx->opt.n_sub;
  const int64_t total = ctx->n_classes * S3;
  const unsigned grid = (unsigned)((total + 127) / 128);
  const double inv_eps2 = 1.0 / (ctx->opt.eps * ctx->opt.eps);
  const Grid<double> gd = device_grid<double>(ctx);
  const bool quad = ctx->opt.basis == kQuad;
  if (ctx->opt.real == MLS_F64) {
    double* t = (double*)ctx->table;
    if (quad)
      k_fast_table<double, kQuad><<<grid, 128, 0, s>>>(gd, ctx->class_axis, ctx->n_classes, ctx->opt.n_sub, inv_eps2, t);
    else
      k_fast_table<double, 4><<<grid, 128, 0, s>>>(gd, ctx->class_axis, ctx->n_classes, ctx->opt.n_sub, inv_eps2, t);
  } else {
    float* t = (float*)ctx->table;
    if (quad)
      k_fast_table<float, kQuad><<<grid, 128, 0, s>>>(gd, ctx->class_axis, ctx->n_classes, ctx->opt.n_sub, inv_eps2, t);
    else
      k_fast_table<float, 4><<<grid, 128, 0, s>>>(gd, ctx->class_axis, ctx->n_classes, ctx->opt.n_sub, inv_eps2, t);
  }
  return cudaGetLastError();
}

}  // namespace mls
