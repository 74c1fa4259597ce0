// Gradients of interpolated fields at the markers from the derivatives of the
// exact-MLS shape functions (Section 2: MLS gives values and spatial
// derivatives; the solver needs velocity and pressure gradients at markers).
#include "transfer_common.cuh"

namespace mls {

// Entry (i, j) of sum_k W_k xi_k,d^extra p~_k p~_k^T from per-axis moments
// S[m][e] = sum_a w_e(a) xi_e,a^m: p~ = [1, xi_x, xi_y, xi_z], so the entry
// is the product over axes e of S[m_e][e] with m_e = [i = e+1] + [j = e+1]
// (+1 on the axis `extra`, or none when extra < 0).
template <typename R>
__device__ __forceinline__ R moment_entry(const R S[4][3], int i, int j, int extra) {
  R v = R(1);
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int m = (i == e + 1) + (j == e + 1) + (e == extra);
    v *= S[m][e];
  }
  return v;
}

// G[c][d][l] = sum_k d_d phi_k^l u_c,k.  One thread per marker in tile
// order.  With the basis centred at the marker, gamma = A^-1 e_0 and
//   d_d phi_k = W_k (alpha_d xi_k,d (p~_k . gamma) + p~_k . A^-1 (e_{d+1}/Delta_d - d_d A gamma)),
// alpha_d = 2 / (eps^2 Delta_d), d_d A = alpha_d sum_k W_k xi_k,d p~_k p~_k^T
// (xi in home-cell widths Delta_d, Gaussian weight).  A and the three d_d A
// are assembled from per-axis moments up to the third; the Cholesky factor of
// A (one refinement step for gamma in single precision) serves all four
// solves.  Markers without support get G = 0.  In single precision the kernel
// is held to 128 registers so two blocks fit per SM: the 81 gathers of a
// marker go straight to the cache hierarchy, and one block per SM (the
// unbounded 142 registers) leaves too few warps to cover them.
template <typename R, typename FT>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 2 : 1)
    k_interp_gradient(Dims D, Grid<R> g, const R* __restrict__ x, const int32_t* __restrict__ home,
                      const int32_t* __restrict__ perm, int64_t M, R inv_eps2, int refine,
                      const FT* __restrict__ u, R* __restrict__ G) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const int64_t m = perm[j];
  const int32_t hc = home[j];
  R out[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) out[c][d] = R(0);
  if (hc >= 0) {
    int i[3];
    decode_home(hc, D, i);
    AxisNodes<R> s[3];
    s[0] = axis_nodes(g.ax[0], i[0], x[m]);
    s[1] = axis_nodes(g.ax[1], i[1], x[M + m]);
    s[2] = axis_nodes(g.ax[2], i[2], x[2 * M + m]);
    R w[3][3], S[4][3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      S[0][e] = S[1][e] = S[2][e] = S[3][e] = R(0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R xi = s[e].xi[a];
        const R wa = dev_exp<R>(-(xi * xi) * inv_eps2);
        w[e][a] = wa;
        S[0][e] += wa;
        S[1][e] += wa * xi;
        S[2][e] += wa * xi * xi;
        S[3][e] += wa * xi * xi * xi;
      }
    }
    const int pi[10] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3};
    const int pj[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
    R A[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) A[q] = moment_entry(S, pi[q], pj[q], -1);
    Chol4<R> ch;
    ch.factor(A);
    if (ch.ok) {
      R gam[4];
      const R e0[4] = {R(1), R(0), R(0), R(0)};
      ch.solve(e0, gam);
      for (int it = 0; it < refine; ++it) {
        R Ay[4], r[4], dy[4];
        sym_mul(A, gam, Ay);
        r[0] = R(1) - Ay[0];
        r[1] = -Ay[1];
        r[2] = -Ay[2];
        r[3] = -Ay[3];
        ch.solve(r, dy);
#pragma unroll
        for (int q = 0; q < 4; ++q) gam[q] += dy[q];
      }
      R alpha[3], dg[3][4];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const R inv_h = R(1) / s[d].w[1];
        alpha[d] = R(2) * inv_eps2 * inv_h;
        R dA[10], v[4], rhs[4];
#pragma unroll
        for (int q = 0; q < 10; ++q) dA[q] = alpha[d] * moment_entry(S, pi[q], pj[q], d);
        sym_mul(dA, gam, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) rhs[q] = (q == d + 1 ? inv_h : R(0)) - v[q];
        ch.solve(rhs, dg[d]);
      }
      int xs[3], ys[3], zs[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        xs[a] = wrap(i[0] + a - 1, D.n[0], D.periodic[0]);
        ys[a] = wrap(i[1] + a - 1, D.n[1], D.periodic[1]);
        zs[a] = wrap(i[2] + a - 1, D.n[2], D.periodic[2]);
      }
      const int64_t N = (int64_t)D.n[0] * D.n[1] * D.n[2];
#pragma unroll
      for (int cz = 0; cz < 3; ++cz)
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) {
          const int64_t row = ((int64_t)zs[cz] * D.n[1] + ys[cy]) * D.n[0];
          const R wyz = w[1][cy] * w[2][cz];
#pragma unroll
          for (int cx = 0; cx < 3; ++cx) {
            const R Wk = w[0][cx] * wyz;
            const R xi[3] = {s[0].xi[cx], s[1].xi[cy], s[2].xi[cz]};
            const R gk = gam[0] + gam[1] * xi[0] + gam[2] * xi[1] + gam[3] * xi[2];
            R dphi[3];
#pragma unroll
            for (int d = 0; d < 3; ++d)
              dphi[d] = Wk * (alpha[d] * xi[d] * gk + dg[d][0] + dg[d][1] * xi[0] + dg[d][2] * xi[1] +
                              dg[d][3] * xi[2]);
            const int64_t o = row + xs[cx];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const R uc = load_field<R, FT>(u + c * N + o);
#pragma unroll
              for (int d = 0; d < 3; ++d) out[c][d] += dphi[d] * uc;
            }
          }
        }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) G[(3 * c + d) * M + m] = out[c][d];
}

cudaError_t launch_interp_gradient(const mls_ctx* ctx, const mls_transfer* T, const void* x, const void* u, void* G,
                                   cudaStream_t s) {
  if (T->M == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((T->M + kBlock - 1) / kBlock);
  const Dims D = dims_of(ctx);
  const double ie2 = 1.0 / (ctx->opt.eps * ctx->opt.eps);
  if (ctx->opt.real == MLS_F64)
    k_interp_gradient<double, double><<<(unsigned)((T->M + kBlockF64 - 1) / kBlockF64), kBlockF64, 0, s>>>(
        D, device_grid<double>(ctx), (const double*)x, T->home, T->perm, T->M, ie2, 0, (const double*)u, (double*)G);
  else if (ctx->opt.field == MLS_F32)
    k_interp_gradient<float, float><<<grid, kBlock, 0, s>>>(D, device_grid<float>(ctx), (const float*)x, T->home,
                                                            T->perm, T->M, (float)ie2, ctx->opt.refine,
                                                            (const float*)u, (float*)G);
  else
    k_interp_gradient<float, __nv_bfloat16><<<grid, kBlock, 0, s>>>(D, device_grid<float>(ctx), (const float*)x,
                                                                    T->home, T->perm, T->M, (float)ie2,
                                                                    ctx->opt.refine, (const __nv_bfloat16*)u,
                                                                    (float*)G);
  return cudaGetLastError();
}

}  // namespace mls
