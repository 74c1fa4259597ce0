// Marker preparation (triangle centroids and areas) and the counting sort
// that groups markers by spreading tile before the build.
#include "mls_host.h"

namespace mls {

// Centroid C = ((V1+V2)+V3)/3 and area |(V2-V1)x(V3-V1)|/2 of triangles
// [t0, t1) of nt, every operation rounded to nearest in R with no contraction,
// so the result is reproducible bit for bit by any IEEE implementation of the
// same order.
template <typename R>
__global__ void __launch_bounds__(kBlock) k_prep(const R* __restrict__ V, int64_t nv,
                                                 const int32_t* __restrict__ tri, int64_t t0, int64_t t1,
                                                 int64_t nt, R* __restrict__ x, R* __restrict__ area) {
  using O = Ops<R>;
  const int64_t t = t0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= t1) return;
  const int64_t i0 = tri[3 * t], i1 = tri[3 * t + 1], i2 = tri[3 * t + 2];
  if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) {
    x[t] = x[nt + t] = x[2 * nt + t] = O::nan_();
    area[t] = O::nan_();
    return;
  }
  R a[3], b[3], c[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    a[d] = V[3 * i0 + d];
    b[d] = V[3 * i1 + d];
    c[d] = V[3 * i2 + d];
  }
  R xc[3], ar;
  triangle_marker(a, b, c, xc, ar);
#pragma unroll
  for (int d = 0; d < 3; ++d) x[d * nt + t] = xc[d];
  area[t] = ar;
}

cudaError_t launch_prep(int real, const void* V, int64_t nv, const int32_t* tri, int64_t t0, int64_t t1,
                        int64_t nt, void* x, void* area, cudaStream_t s) {
  if (t1 <= t0) return cudaSuccess;
  const unsigned grid = (unsigned)((t1 - t0 + kBlock - 1) / kBlock);
  if (real == MLS_F64)
    k_prep<double><<<grid, kBlock, 0, s>>>((const double*)V, nv, tri, t0, t1, nt, (double*)x, (double*)area);
  else
    k_prep<float><<<grid, kBlock, 0, s>>>((const float*)V, nv, tri, t0, t1, nt, (float*)x, (float*)area);
  return cudaGetLastError();
}

// Markers per thread of the locate and scatter kernels: 4 on workloads that
// fill the GPU several times over (their loads then overlap), 1 on small ones
// (which need every block they can get).
constexpr int kLocatePer = 4;
inline int locate_per(int64_t M) { return M >= (int64_t)kLocatePer * 152 * 2048 ? kLocatePer : 1; }

// Triangles whose markers the locate kernel forms itself (the preparation
// fused into it): vertices, their count, the triangles, and where the
// markers' positions and areas go.
template <typename R>
struct PrepSource {
  const R* V;
  int64_t nv;
  const int32_t* tri;
  R* x;
  R* area;
};

// Home cell of markers [j0, j1) of M, their spreading-tile bins, and their
// ranks inside the bins (warp-aggregated atomic counter per bin).  Dropped
// markers go to the last bin and are counted in status[0] (all) and
// status[1] (non-finite).  With PREP the markers are first formed from their
// triangles as by k_prep (same operations, same NaN rule) and stored.
template <typename R, int PER, bool PREP>
__global__ void __launch_bounds__(kBlock) k_locate(Grid<R> g, Tiles tl, const R* __restrict__ x,
                                                   const R* __restrict__ area, int64_t M, int64_t j0, int64_t j1,
                                                   PrepSource<R> src, int32_t* __restrict__ key,
                                                   int32_t* __restrict__ rank, int32_t* __restrict__ counts,
                                                   unsigned long long* __restrict__ status,
                                                   int32_t* __restrict__ sub) {
  // A warp takes PER rounds of 32 consecutive markers; every round's
  // loads, then every round's bin counter update, are issued before any
  // result is waited for.
  const int lane = threadIdx.x & 31;
  const int64_t w0 = j0 + ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 * PER);
  R p[PER][3], ar[PER];
  if constexpr (PREP) {
    using O = Ops<R>;
    int64_t iv[PER][3];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int64_t j = w0 + r * 32 + lane;
      if (j < j1) {
#pragma unroll
        for (int q = 0; q < 3; ++q) iv[r][q] = src.tri[3 * j + q];
      }
    }
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int64_t j = w0 + r * 32 + lane;
      if (j < j1) {
        const int64_t i0 = iv[r][0], i1 = iv[r][1], i2 = iv[r][2];
        if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= src.nv || i1 >= src.nv || i2 >= src.nv) {
          p[r][0] = p[r][1] = p[r][2] = ar[r] = O::nan_();
        } else {
          R va[3], vb[3], vc[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            va[d] = src.V[3 * i0 + d];
            vb[d] = src.V[3 * i1 + d];
            vc[d] = src.V[3 * i2 + d];
          }
          triangle_marker(va, vb, vc, p[r], ar[r]);
        }
        src.x[j] = p[r][0];
        src.x[M + j] = p[r][1];
        src.x[2 * M + j] = p[r][2];
        src.area[j] = ar[r];
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int64_t j = w0 + r * 32 + lane;
      if (j < j1) {
        p[r][0] = x[j];
        p[r][1] = x[M + j];
        p[r][2] = x[2 * M + j];
        ar[r] = area[j];
      }
    }
  }
  int k[PER], cell[PER];
  unsigned peers[PER];
  int base[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int64_t j = w0 + r * 32 + lane;
    k[r] = -1;   // no marker: a group of its own that counts nothing
    cell[r] = 0;
    if (j < j1) {
      const bool finite = isfinite(p[r][0]) && isfinite(p[r][1]) && isfinite(p[r][2]) && isfinite(ar[r]);
      bool ok = finite;
      int h[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        h[d] = locate_axis(g.ax[d], p[r][d]);
        ok = ok && support_ok(g.ax[d], h[d]);
      }
      k[r] = tl.nbins - 1;
      if (ok) {
        k[r] = (((h[2] >> tl.l[2]) * tl.nb[1]) + (h[1] >> tl.l[1])) * tl.nb[0] + (h[0] >> tl.l[0]);
        cell[r] = ((((h[2] & ((1 << tl.l[2]) - 1)) << tl.l[1]) | (h[1] & ((1 << tl.l[1]) - 1))) << tl.l[0]) |
                  (h[0] & ((1 << tl.l[0]) - 1));
      } else {
        atomicAdd(&status[0], 1ULL);
        if (!finite) atomicAdd(&status[1], 1ULL);
      }
    }
    peers[r] = __match_any_sync(0xffffffffu, k[r]);
    base[r] = 0;
    if (k[r] >= 0 && lane == __ffs(peers[r]) - 1) base[r] = atomicAdd(&counts[k[r]], __popc(peers[r]));
  }
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int64_t j = w0 + r * 32 + lane;
    const int b = __shfl_sync(0xffffffffu, base[r], __ffs(peers[r]) - 1);
    if (j < j1) {
      key[j] = k[r];
      rank[j] = b + __popc(peers[r] & ((1u << lane) - 1u));
      if (sub && k[r] != tl.nbins - 1) sub[j] = cell[r];
    }
  }
}

// The in-tile sort by home cell runs when a tile has at most kSortCells cells.
// Until the build overwrites them, three of the transfer's output arrays
// serve it as scratch: the first plane of phi holds each marker's cell
// inside its tile (caller order), home the unsorted tile order and c (as
// int32) the cells in that order.
bool tile_sort_on(const mls_ctx* ctx) {
  return ctx->tiles.l[0] + ctx->tiles.l[1] + ctx->tiles.l[2] <= kSortCellsLog2;
}

template <typename R>
static void locate_range(const mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M,
                         int64_t j0, int64_t j1, PrepSource<R> src, bool prep, cudaStream_t s) {
  const int64_t n = j1 - j0;
  const int per = locate_per(n);
  const unsigned grid = (unsigned)((n + kBlock * per - 1) / (kBlock * per));
  int32_t* sub = tile_sort_on(ctx) ? reinterpret_cast<int32_t*>(T->phi) : nullptr;
  auto kern = prep ? (per == kLocatePer ? k_locate<R, kLocatePer, true> : k_locate<R, 1, true>)
                   : (per == kLocatePer ? k_locate<R, kLocatePer, false> : k_locate<R, 1, false>);
  kern<<<grid, kBlock, 0, s>>>(device_grid<R>(ctx), ctx->tiles, (const R*)x, (const R*)area, M, j0, j1, src, T->key,
                               T->rank, T->counts, T->status, sub);
}

cudaError_t launch_locate(const mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M,
                          cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  if (ctx->opt.real == MLS_F64)
    locate_range<double>(ctx, T, x, area, M, 0, M, PrepSource<double>{}, false, s);
  else
    locate_range<float>(ctx, T, x, area, M, 0, M, PrepSource<float>{}, false, s);
  return cudaGetLastError();
}

cudaError_t launch_prep_locate(const mls_ctx* ctx, mls_transfer* T, const void* V, int64_t nv, const int32_t* tri,
                               int64_t nt, int64_t t0, int64_t t1, void* x, void* area, cudaStream_t s) {
  if (t1 <= t0) return cudaSuccess;
  if (ctx->opt.real == MLS_F64)
    locate_range<double>(ctx, T, nullptr, nullptr, nt, t0, t1,
                         PrepSource<double>{(const double*)V, nv, tri, (double*)x, (double*)area}, true, s);
  else
    locate_range<float>(ctx, T, nullptr, nullptr, nt, t0, t1,
                        PrepSource<float>{(const float*)V, nv, tri, (float*)x, (float*)area}, true, s);
  return cudaGetLastError();
}

// ---- exclusive scan of the bin counts (three passes, no inter-block waits) ----

constexpr int kScanThreads = 512;
constexpr int kScanPer = kScanTile / kScanThreads;  // 8 bins per thread

__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_tot, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int w = lane < nw ? warp_tot[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int n = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += n;
    }
    if (lane < nw) warp_tot[lane] = wi - w;
    if (lane == nw - 1) *total = wi;
  }
  __syncthreads();
  return incl - v + warp_tot[wid];
}

// Per scan tile of 4096 bins: the number of markers and the number of
// non-empty spreading tiles (the last bin, dropped markers, is not a tile).
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t* __restrict__ counts, int nbins,
                                                              int ntiles, int32_t* __restrict__ tile_sums) {
  __shared__ int warp_tot[32];
  __shared__ int total;
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  int v = 0, ne = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q)
    if (base + q < nbins) {
      const int cq = counts[base + q];
      v += cq;
      ne += (cq > 0 && base + q < nbins - 1) ? 1 : 0;
    }
  block_exclusive_scan(v, warp_tot, &total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
  __syncthreads();
  block_exclusive_scan(ne, warp_tot, &total);
  if (threadIdx.x == 0) tile_sums[ntiles + blockIdx.x] = total;
}

// Bin offsets (exclusive prefix of the counts) and the ascending list of
// non-empty spreading tiles.  Each block first sums the per-scan-tile totals
// of the blocks before it (at most kScanMaxTiles values); the last block also
// writes the length of the tile list.
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int32_t* __restrict__ counts, int nbins, int ntiles,
                                                             const int32_t* __restrict__ tile_sums,
                                                             int32_t* __restrict__ offsets,
                                                             int32_t* __restrict__ items,
                                                             int32_t* __restrict__ n_items) {
  __shared__ int warp_tot[32];
  __shared__ int total;
  int pc = 0, pi = 0;
  for (int t = threadIdx.x; t < (int)blockIdx.x; t += kScanThreads) {
    pc += tile_sums[t];
    pi += tile_sums[ntiles + t];
  }
  block_exclusive_scan(pc, warp_tot, &total);
  const int prefix_c = total;
  __syncthreads();
  block_exclusive_scan(pi, warp_tot, &total);
  const int prefix_i = total;
  __syncthreads();
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  int v[kScanPer];
  int s = 0, ne = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    v[q] = base + q < nbins ? counts[base + q] : 0;
    s += v[q];
    ne += (v[q] > 0 && base + q < nbins - 1) ? 1 : 0;
  }
  int run = block_exclusive_scan(s, warp_tot, &total) + prefix_c;
  __syncthreads();
  int pos = block_exclusive_scan(ne, warp_tot, &total) + prefix_i;
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *n_items = prefix_i + total;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    if (base + q < nbins) {
      offsets[base + q] = run;
      if (v[q] > 0 && base + q < nbins - 1) items[pos++] = base + q;
    }
    run += v[q];
  }
}

cudaError_t launch_scan(mls_transfer* T, int nbins, cudaStream_t s, mls_ctx* ctx) {
  const int ntiles = (nbins + kScanTile - 1) / kScanTile;
  int slot = timer_begin(ctx, "scan_reduce", s);
  k_scan_reduce<<<ntiles, kScanThreads, 0, s>>>(T->counts, nbins, ntiles, T->tile_sums);
  timer_end(ctx, slot, s);
  slot = timer_begin(ctx, "scan_apply", s);
  k_scan_apply<<<ntiles, kScanThreads, 0, s>>>(T->counts, nbins, ntiles, T->tile_sums, T->offsets, T->items,
                                               T->n_items);
  timer_end(ctx, slot, s);
  return cudaGetLastError();
}

// perm[offsets[bin] + rank] = caller index: stable within nothing, grouped by
// bin.  With the in-tile sort, the caller index and the marker's cell in its
// tile go to the sort's scratch arrays instead (`perm` unsorted, `cell`).
template <int PER>
__global__ void __launch_bounds__(kBlock) k_scatter(const int32_t* __restrict__ key, const int32_t* __restrict__ rank,
                                                    const int32_t* __restrict__ offsets, int64_t M,
                                                    int32_t* __restrict__ perm, const int32_t* __restrict__ sub,
                                                    int32_t* __restrict__ cell) {
  // PER markers per thread, a block's in consecutive strides, so that
  // the loads of all of them are in flight before the first store.
  const int64_t j0 = (int64_t)blockIdx.x * blockDim.x * PER + threadIdx.x;
  int64_t pos[PER];
  int cl[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int64_t j = j0 + (int64_t)r * blockDim.x;
    pos[r] = -1;
    if (j < M) {
      pos[r] = offsets[key[j]] + rank[j];
      if (cell) cl[r] = sub[j];
    }
  }
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int64_t j = j0 + (int64_t)r * blockDim.x;
    if (pos[r] >= 0) {
      perm[pos[r]] = (int32_t)j;
      if (cell) cell[pos[r]] = cl[r];
    }
  }
}

cudaError_t launch_scatter(const mls_ctx* ctx, mls_transfer* T, int64_t M, cudaStream_t s) {
  const int per = locate_per(M);
  const unsigned grid = (unsigned)((M + kBlock * per - 1) / (kBlock * per));
  auto k = per == kLocatePer ? k_scatter<kLocatePer> : k_scatter<1>;
  if (tile_sort_on(ctx))
    k<<<grid, kBlock, 0, s>>>(T->key, T->rank, T->offsets, M, T->home, reinterpret_cast<const int32_t*>(T->phi),
                              reinterpret_cast<int32_t*>(T->c));
  else
    k<<<grid, kBlock, 0, s>>>(T->key, T->rank, T->offsets, M, T->perm, nullptr, nullptr);
  return cudaGetLastError();
}

// Orders the markers of each spreading tile by home cell (counting sort over
// the tile's cells), so that markers sharing a home cell, and so their 27
// support nodes, are adjacent in tile order; the order inside one cell is
// not fixed.  One warp per tile with a private histogram in shared memory
// (one padding word after every 32 bins, so that the scan's lanes, each
// owning a run of consecutive bins, read 32 different banks): count,
// exclusive scan, then each marker takes the next place of its cell.
// The dropped markers (last bin) keep their places.
__global__ void __launch_bounds__(kSortThreads) k_tile_sort(Tiles tl, const int32_t* __restrict__ items,
                                                            const int32_t* __restrict__ n_items_p,
                                                            const int32_t* __restrict__ offsets,
                                                            const int32_t* __restrict__ counts, int64_t M,
                                                            const int32_t* __restrict__ perm0,
                                                            const int32_t* __restrict__ cell,
                                                            int32_t* __restrict__ perm) {
  extern __shared__ int hist_all[];
  const int C = 1 << (tl.l[0] + tl.l[1] + tl.l[2]);
  const int lane = threadIdx.x & 31;
  int* hist = hist_all + (threadIdx.x >> 5) * (C + (C >> 5));
  const int per = (C + 31) >> 5;          // bins per lane in the scan
  const int lo = min(C, lane * per), hi = min(C, lo + per);
  const int n_items = *n_items_p;
  const int warps = gridDim.x * (kSortThreads / 32);
  for (int it = blockIdx.x * (kSortThreads / 32) + (threadIdx.x >> 5); it < n_items; it += warps) {
    const int b = items[it];
    const int s = offsets[b], n = counts[b];
    if (n == 1) {
      if (lane == 0) perm[s] = perm0[s];
      continue;
    }
    for (int q = lane; q < C + (C >> 5); q += 32) hist[q] = 0;
    __syncwarp();
    // Windows of 256 markers: the eight loads of a lane are issued together.
    for (int w0 = 0; w0 < n; w0 += 256) {
      int cw[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = w0 + u * 32 + lane;
        cw[u] = i < n ? cell[s + i] : -1;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (cw[u] >= 0) atomicAdd(&hist[cw[u] + (cw[u] >> 5)], 1);
    }
    __syncwarp();
    int sum = 0;
    for (int q = lo; q < hi; ++q) sum += hist[q + (q >> 5)];
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    int run = incl - sum;
    for (int q = lo; q < hi; ++q) {
      const int v = hist[q + (q >> 5)];
      hist[q + (q >> 5)] = run;
      run += v;
    }
    __syncwarp();
    for (int w0 = 0; w0 < n; w0 += 256) {
      int cw[8], pw[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = w0 + u * 32 + lane;
        cw[u] = i < n ? cell[s + i] : -1;
        pw[u] = i < n ? perm0[s + i] : 0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (cw[u] >= 0) perm[s + atomicAdd(&hist[cw[u] + (cw[u] >> 5)], 1)] = pw[u];
    }
    __syncwarp();
  }
  const int64_t d0 = offsets[tl.nbins - 1];
  for (int64_t j = d0 + (int64_t)blockIdx.x * kSortThreads + threadIdx.x; j < M;
       j += (int64_t)gridDim.x * kSortThreads)
    perm[j] = perm0[j];
}

cudaError_t launch_tile_sort(const mls_ctx* ctx, mls_transfer* T, int64_t M, cudaStream_t s) {
  if (!tile_sort_on(ctx)) return cudaSuccess;
  const int C = 1 << (ctx->tiles.l[0] + ctx->tiles.l[1] + ctx->tiles.l[2]);
  const size_t smem = (size_t)(kSortThreads / 32) * (C + (C >> 5)) * 4;
  k_tile_sort<<<ctx->sort_grid, kSortThreads, smem, s>>>(ctx->tiles, T->items, T->n_items, T->offsets, T->counts, M,
                                                          T->home, reinterpret_cast<const int32_t*>(T->c), T->perm);
  return cudaGetLastError();
}

cudaError_t sort_configure(mls_ctx* ctx) {
  ctx->sort_grid = 0;
  if (!tile_sort_on(ctx)) return cudaSuccess;
  const int C = 1 << (ctx->tiles.l[0] + ctx->tiles.l[1] + ctx->tiles.l[2]);
  const int smem = (kSortThreads / 32) * (C + (C >> 5)) * 4;
  cudaError_t e = raise_smem_limit((const void*)k_tile_sort, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0, dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_sort, kSortThreads, smem)) != cudaSuccess)
    return e;
  ctx->sort_grid = (per_sm > 0 ? per_sm : 1) * sms;
  return cudaSuccess;
}

}  // namespace mls
