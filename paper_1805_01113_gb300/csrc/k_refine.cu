// Adaptive Lagrangian refinement of the forcing markers (Section 3, Fig. 5):
// base triangles split into 1, 2, 3 or 4 triangles for the forcing step, the
// level chosen from the element size against the local grid spacing.
#include <algorithm>
#include <cmath>

#include "mls_host.h"

namespace mls {

constexpr int kRefineThreads = 256;

struct RefineArgs {
  const void* V;
  int64_t nv;
  const int32_t* tri;
  int64_t nt;
  double ratio;
  double length2_per_area;  // 4 / sqrt(3): l^2 of the equilateral triangle of unit area
  int max_level;
  int32_t* level;           // [nt]
  int32_t* local;           // [nt] offset inside the block
  int64_t* block_sum;       // [blocks] pieces per block, then their exclusive prefix
  int64_t* total;           // [1]
};

template <typename R>
__device__ __forceinline__ bool load_triangle(const RefineArgs& a, int64_t t, R v[3][3]) {
  const R* V = static_cast<const R*>(a.V);
  const int64_t i0 = a.tri[3 * t], i1 = a.tri[3 * t + 1], i2 = a.tri[3 * t + 2];
  if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= a.nv || i1 >= a.nv || i2 >= a.nv) return false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    v[0][d] = V[3 * i0 + d];
    v[1][d] = V[3 * i1 + d];
    v[2][d] = V[3 * i2 + d];
  }
  return true;
}

// Level of each base triangle: the smallest k <= max_level with
// l^2 / (k + 1) <= (ratio h)^2, l^2 = 4 A / sqrt(3) from the triangle's
// (working-precision) area, h the smallest width of the home cell of its
// centroid, compared in double precision; level 0 for a centroid outside the
// grid or a triangle with an invalid vertex index.  Also the exclusive scan
// of the pieces (k + 1) inside each block.
template <typename R>
__global__ void __launch_bounds__(kRefineThreads) k_refine_plan(RefineArgs a, Grid<R> g, Grid<double> gd) {
  const int64_t t = (int64_t)blockIdx.x * kRefineThreads + threadIdx.x;
  int pieces = 0;
  if (t < a.nt) {
    int lev = 0;
    R v[3][3];
    if (load_triangle(a, t, v)) {
      R xc[3], area;
      triangle_marker(v[0], v[1], v[2], xc, area);
      bool inside = true;
      double h = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int i = locate_axis(g.ax[d], xc[d]);
        inside = inside && i >= 0;
        const double w = i >= 0 ? gd.ax[d].widths[i] : 0.0;
        h = d == 0 ? w : fmin(h, w);
      }
      if (inside && isfinite((double)area)) {
        const double s = __dmul_rn((double)area, a.length2_per_area);
        const double rh = __dmul_rn(a.ratio, h);
        const double tt = __dmul_rn(rh, rh);
        lev = a.max_level;
        for (int k = a.max_level; k >= 0; --k)
          if (s <= __dmul_rn((double)(k + 1), tt)) lev = k;
      }
    }
    a.level[t] = lev;
    pieces = lev + 1;
  }
  // Block-wide exclusive scan of the pieces.
  __shared__ int warp_tot[kRefineThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = pieces;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < kRefineThreads / 32 ? warp_tot[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += n;
    }
    if (lane < kRefineThreads / 32) warp_tot[lane] = wi - w;
    if (lane == kRefineThreads / 32 - 1) a.block_sum[blockIdx.x] = wi;
  }
  __syncthreads();
  if (t < a.nt) a.local[t] = incl - pieces + warp_tot[wid];
}

// Exclusive prefix of the block sums (one block, strided), and the total.
__global__ void __launch_bounds__(1024) k_refine_scan(int64_t* __restrict__ block_sum, int nb,
                                                      int64_t* __restrict__ total) {
  __shared__ int64_t part[1024];
  const int tid = threadIdx.x;
  const int per = (nb + 1023) / 1024;
  const int b0 = tid * per, b1 = min(nb, b0 + per);
  int64_t s = 0;
  for (int b = b0; b < b1; ++b) s += block_sum[b];
  part[tid] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int64_t v = tid >= o ? part[tid - o] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int64_t run = part[tid] - s;
  for (int b = b0; b < b1; ++b) {
    const int64_t v = block_sum[b];
    block_sum[b] = run;
    run += v;
  }
  if (tid == 1023) *total = part[1023];
}

// Refined markers: the triangles of Fig. 5 for the triangle's level, in the
// order (level 1) (V1, L1, V3), (L1, V2, V3); (level 2) (V1, V2, L2),
// (V2, V3, L2), (V3, V1, L2); (level 3) (V1, L31, L33), (L31, V2, L32),
// (L33, L32, V3), (L31, L32, L33), with L1 = L31 = (V1+V2)/2,
// L32 = (V2+V3)/2, L33 = (V3+V1)/2 and L2 = ((V1+V2)+V3)/3; each gives the
// centroid and area of a base marker.  Markers past `capacity` are not
// written (the host reports MLS_ERR_CAPACITY).
template <typename R>
__global__ void __launch_bounds__(kRefineThreads) k_refine_emit(RefineArgs a, int64_t capacity, R* __restrict__ x,
                                                                R* __restrict__ area, int32_t* __restrict__ parent) {
  using O = Ops<R>;
  const int64_t t = (int64_t)blockIdx.x * kRefineThreads + threadIdx.x;
  if (t >= a.nt) return;
  const int lev = a.level[t];
  const int64_t off = a.block_sum[blockIdx.x] + a.local[t];
  if (off + lev + 1 > capacity) return;
  R v[3][3];
  if (!load_triangle(a, t, v)) {
    x[off] = x[capacity + off] = x[2 * capacity + off] = O::nan_();
    area[off] = O::nan_();
    parent[off] = (int32_t)t;
    return;
  }
  R p[4][3][3];  // up to four triangles, three points each
  int np = 1;
  if (lev == 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      p[0][0][d] = v[0][d];
      p[0][1][d] = v[1][d];
      p[0][2][d] = v[2][d];
    }
  } else if (lev == 1) {
    np = 2;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const R l1 = O::mul(O::add(v[0][d], v[1][d]), R(0.5));
      p[0][0][d] = v[0][d];
      p[0][1][d] = l1;
      p[0][2][d] = v[2][d];
      p[1][0][d] = l1;
      p[1][1][d] = v[1][d];
      p[1][2][d] = v[2][d];
    }
  } else if (lev == 2) {
    np = 3;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const R l2 = O::div(O::add(O::add(v[0][d], v[1][d]), v[2][d]), R(3));
      p[0][0][d] = v[0][d];
      p[0][1][d] = v[1][d];
      p[0][2][d] = l2;
      p[1][0][d] = v[1][d];
      p[1][1][d] = v[2][d];
      p[1][2][d] = l2;
      p[2][0][d] = v[2][d];
      p[2][1][d] = v[0][d];
      p[2][2][d] = l2;
    }
  } else {
    np = 4;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const R l31 = O::mul(O::add(v[0][d], v[1][d]), R(0.5));
      const R l32 = O::mul(O::add(v[1][d], v[2][d]), R(0.5));
      const R l33 = O::mul(O::add(v[2][d], v[0][d]), R(0.5));
      p[0][0][d] = v[0][d];
      p[0][1][d] = l31;
      p[0][2][d] = l33;
      p[1][0][d] = l31;
      p[1][1][d] = v[1][d];
      p[1][2][d] = l32;
      p[2][0][d] = l33;
      p[2][1][d] = l32;
      p[2][2][d] = v[2][d];
      p[3][0][d] = l31;
      p[3][1][d] = l32;
      p[3][2][d] = l33;
    }
  }
  for (int q = 0; q < np; ++q) {
    R xc[3], ar;
    triangle_marker(p[q][0], p[q][1], p[q][2], xc, ar);
    const int64_t o = off + q;
    x[o] = xc[0];
    x[capacity + o] = xc[1];
    x[2 * capacity + o] = xc[2];
    area[o] = ar;
    parent[o] = (int32_t)t;
  }
}

int64_t refine_workspace_bytes(int64_t nt) {
  const int64_t nb = (nt + kRefineThreads - 1) / kRefineThreads;
  return 2 * 4 * nt + 8 * nb + 8 + 64;
}

cudaError_t launch_refine(const mls_ctx* ctx, const void* V, int64_t nv, const int32_t* tri, int64_t nt,
                          double ratio, int max_level, int64_t capacity, void* x, void* area, int32_t* parent,
                          int32_t* level, void* ws, int64_t* total_host, cudaStream_t s) {
  const int64_t nb = (nt + kRefineThreads - 1) / kRefineThreads;
  RefineArgs a;
  a.V = V;
  a.nv = nv;
  a.tri = tri;
  a.nt = nt;
  a.ratio = ratio;
  a.length2_per_area = 4.0 / std::sqrt(3.0);
  a.max_level = max_level;
  char* w = static_cast<char*>(ws);
  a.local = reinterpret_cast<int32_t*>(w);
  a.level = level ? level : reinterpret_cast<int32_t*>(w + 4 * nt);
  a.block_sum = reinterpret_cast<int64_t*>(w + ((8 * nt + 7) & ~int64_t(7)));
  a.total = a.block_sum + nb;
  cudaError_t e;
  if (ctx->opt.real == MLS_F64)
    k_refine_plan<double><<<(unsigned)nb, kRefineThreads, 0, s>>>(a, device_grid<double>(ctx), device_grid<double>(ctx));
  else
    k_refine_plan<float><<<(unsigned)nb, kRefineThreads, 0, s>>>(a, device_grid<float>(ctx), device_grid<double>(ctx));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_refine_scan<<<1, 1024, 0, s>>>(a.block_sum, (int)nb, a.total);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ctx->opt.real == MLS_F64)
    k_refine_emit<double><<<(unsigned)nb, kRefineThreads, 0, s>>>(a, capacity, (double*)x, (double*)area, parent);
  else
    k_refine_emit<float><<<(unsigned)nb, kRefineThreads, 0, s>>>(a, capacity, (float*)x, (float*)area, parent);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(total_host, a.total, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

}  // namespace mls
