// Euler-to-Lagrange interpolation (gather) and Lagrange-to-Euler spreading
// (scatter through shared-memory tile accumulators in single precision,
// direct global reductions in double precision).
#include <type_traits>

#include "transfer_common.cuh"

namespace mls {

// U_l = sum_k phi_k^l u_k for the 3 components (text after Eq. 6), double
// precision.  One thread per stored marker; the 27 phi values are read with
// unit stride across the warp, the field through the read-only path.
template <typename R, typename FT>
__global__ void __launch_bounds__(kBlock) k_interp(Dims D, const R* __restrict__ phi, const int32_t* __restrict__ home,
                                                   const int32_t* __restrict__ perm, int64_t M, int64_t cap,
                                                   const FT* __restrict__ u, R* __restrict__ U) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const int64_t m = perm[j];
  const int32_t h = home[j];
  if (h < 0) {
    U[m] = R(0);
    U[M + m] = R(0);
    U[2 * M + m] = R(0);
    return;
  }
  int i[3];
  decode_home(h, D, i);
  int xs[3], ys[3], zs[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    xs[a] = wrap(i[0] + a - 1, D.n[0], D.periodic[0]);
    ys[a] = wrap(i[1] + a - 1, D.n[1], D.periodic[1]);
    zs[a] = wrap(i[2] + a - 1, D.n[2], D.periodic[2]);
  }
  const int64_t N = (int64_t)D.n[0] * D.n[1] * D.n[2];
  R s0 = R(0), s1 = R(0), s2 = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int64_t row = ((int64_t)zs[c] * D.n[1] + ys[b]) * D.n[0];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const R p = phi[(9 * c + 3 * b + a) * cap + j];
        const int64_t o = row + xs[a];
        s0 += p * load_field<R, FT>(u + o);
        s1 += p * load_field<R, FT>(u + N + o);
        s2 += p * load_field<R, FT>(u + 2 * N + o);
      }
    }
  U[m] = s0;
  U[M + m] = s1;
  U[2 * M + m] = s2;
}

// U_l = sum_k phi_k^l u_k (text after Eq. 6), single precision, by spreading
// tile.  Persistent blocks walk the non-empty tiles; for a tile each marker
// flags the 9 brick rows (y, z) its support touches, the block copies the
// flagged rows of the three field components into shared memory with
// asynchronous copies, then each thread gathers its markers' 27 x 3 values
// from shared memory.  Blocks then zero U of the dropped markers (the last
// bin of the tile sort).  A float brick is copied cell by cell; a bfloat16
// brick keeps the 2-byte values and is copied in 4-byte pairs of cells when
// the field allows it (`pairs`: an even x extent and a 4-byte aligned field),
// else cell by cell through registers.
template <typename FT, int LX>
__global__ void __launch_bounds__(kInterpThreads) k_interp_brick(
    Dims D, Tiles tl, const float* __restrict__ phi, const int32_t* __restrict__ home,
    const int32_t* __restrict__ perm, const int32_t* __restrict__ items, const int32_t* __restrict__ n_items_p,
    const int32_t* __restrict__ offsets, const int32_t* __restrict__ counts, int64_t M, int64_t cap,
    const FT* __restrict__ u, float* __restrict__ U, int pairs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool BF = sizeof(FT) == 2;
  constexpr int XL = BF ? 2 : 1;                 // halo cells left of the tile in a brick row
  constexpr int BX = (1 << LX) + 2 * XL;
  using BT = typename std::conditional<BF, __nv_bfloat16, float>::type;
  const InterpSmem L(LX, tl.l[1], tl.l[2], BF);
  const int BY = L.BY, PS = L.PS, CELLS = L.CELLS, ROWS = L.ROWS;
  BT* su = reinterpret_cast<BT*>(smem_raw);
  int* row_s = reinterpret_cast<int*>(smem_raw + L.rows);
  int* row_g = row_s + ROWS;
  unsigned char* flag = reinterpret_cast<unsigned char*>(row_g + ROWS);
  const int tid = threadIdx.x;
  const int64_t N = (int64_t)D.n[0] * D.n[1] * D.n[2];
  const int n_items = *n_items_p;
  for (int r = tid; r < ROWS; r += kInterpThreads) flag[r] = 0;
  __syncthreads();
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int b = items[it];
    const int start = offsets[b], end = start + counts[b];
    const int bx = b % tl.nb[0], by = (b / tl.nb[0]) % tl.nb[1], bz = b / (tl.nb[0] * tl.nb[1]);
    const int ox = bx << LX, oy = by << tl.l[1], oz = bz << tl.l[2];
    for (int j = start + tid; j < end; j += kInterpThreads) {
      int i[3];
      decode_home(home[j], D, i);
      const int r0 = (i[2] - oz) * BY + (i[1] - oy);
#pragma unroll
      for (int cz = 0; cz < 3; ++cz)
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) flag[r0 + cz * BY + cy] = 1;
    }
    for (int r = tid; r < ROWS; r += kInterpThreads) {
      const int ey = r % BY, ez = r / BY;
      row_s[r] = ez * PS + ey * BX;
      row_g[r] = wrap(oz - 1 + ez, D.n[2], D.periodic[2]) * D.n[1] + wrap(oy - 1 + ey, D.n[1], D.periodic[1]);
    }
    __syncthreads();
    if constexpr (BF) {
      if (pairs) {
        // Pairs of cells [ox - 2 + 2k, ox - 1 + 2k]: even starts, so with an even
        // x extent a wrapped pair stays a pair and never straddles the last cell.
        constexpr int BP = BX / 2;
        for (int e = tid; e < ROWS * BP; e += kInterpThreads) {
          const int r = e / BP, k = e - r * BP;
          if (!flag[r]) continue;
          int gx = ox - XL + 2 * k;
          if (gx < 0 || gx >= D.n[0]) {
            if (!D.periodic[0]) continue;             // outside a walled axis: never gathered
            gx = gx < 0 ? gx + D.n[0] : gx - D.n[0];
            if (gx < 0 || gx >= D.n[0]) continue;     // beyond one period: never gathered
          }
          const int64_t o = (int64_t)row_g[r] * D.n[0] + gx;
          BT* d = su + row_s[r] + 2 * k;
          cp_async4_pair(d, u + o);
          cp_async4_pair(d + CELLS, u + N + o);
          cp_async4_pair(d + 2 * CELLS, u + 2 * N + o);
        }
      } else {
        for (int e = tid; e < ROWS * BX; e += kInterpThreads) {
          const int r = e / BX, ex = e - r * BX;
          if (!flag[r]) continue;
          int gx = ox - XL + ex;
          if ((gx < 0 || gx >= D.n[0]) && !D.periodic[0]) continue;
          gx = wrap(gx, D.n[0], D.periodic[0]);
          if (gx < 0 || gx >= D.n[0]) continue;
          const int64_t o = (int64_t)row_g[r] * D.n[0] + gx;
          BT* d = su + row_s[r] + ex;
          d[0] = u[o];
          d[CELLS] = u[N + o];
          d[2 * CELLS] = u[2 * N + o];
        }
      }
    } else {
      for (int e = tid; e < ROWS * BX; e += kInterpThreads) {
        const int r = e / BX, ex = e - r * BX;
        if (!flag[r]) continue;
        const int gx = wrap(ox - XL + ex, D.n[0], D.periodic[0]);
        stage_cell(reinterpret_cast<float*>(su) + row_s[r] + ex, CELLS, reinterpret_cast<const float*>(u), N,
                   (int64_t)row_g[r] * D.n[0] + gx);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    for (int r = tid; r < ROWS; r += kInterpThreads) flag[r] = 0;
    for (int j = start + tid; j < end; j += kInterpThreads) {
      int i[3];
      decode_home(home[j], D, i);
      const int base = (i[2] - oz) * PS + (i[1] - oy) * BX + (i[0] - ox) + (XL - 1);
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
      for (int cz = 0; cz < 3; ++cz)
#pragma unroll
        for (int cy = 0; cy < 3; ++cy)
#pragma unroll
          for (int cx = 0; cx < 3; ++cx) {
            const float p = phi[(9 * cz + 3 * cy + cx) * cap + j];
            const int si = base + cz * PS + cy * BX + cx;
            s0 += p * to_f<BT>(su[si]);
            s1 += p * to_f<BT>(su[CELLS + si]);
            s2 += p * to_f<BT>(su[2 * CELLS + si]);
          }
      const int64_t m = perm[j];
      U[m] = s0;
      U[M + m] = s1;
      U[2 * M + m] = s2;
    }
    __syncthreads();
  }
  // Dropped markers (last bin) interpolate to zero.
  const int64_t d0 = offsets[tl.nbins - 1];
  for (int64_t j = d0 + (int64_t)blockIdx.x * kInterpThreads + tid; j < M; j += (int64_t)gridDim.x * kInterpThreads) {
    const int64_t m = perm[j];
    U[m] = 0.f;
    U[M + m] = 0.f;
    U[2 * M + m] = 0.f;
  }
}

template <typename FT>
static const void* interp_kernel(int lx) {
  switch (lx) {
    case 1: return (const void*)k_interp_brick<FT, 1>;
    case 2: return (const void*)k_interp_brick<FT, 2>;
    case 3: return (const void*)k_interp_brick<FT, 3>;
    case 4: return (const void*)k_interp_brick<FT, 4>;
    default: return (const void*)k_interp_brick<FT, 5>;
  }
}

// f_k += sum_l c_l phi_k^l F_l (text after Eq. 7), single precision.
// Persistent blocks walk the list of non-empty spreading tiles, taking up to
// 128 markers of a tile at a time (one per thread).  For such a chunk a block
// finds, per component, the largest |c_l F_l| and scales contributions by a
// power of two so that any |phi| <= 1/2 term is at most 2^22 units, rounds
// them to integers and adds them into a shared-memory accumulator with native
// 32-bit integer atomics; a cell's sum stays below 128 * 2^22 = 2^29.  A
// marker with some |phi| > 1/2 (rare for MLS) adds those terms to f directly
// with float atomics.  Each marker flags the 9 accumulator rows its support
// touches; only flagged rows are converted back, added to f with one global
// atomic per component and cell (per 4 cells with VEC), and reset to zero.
// The quantum is at most 2^-22 of the chunk's largest |c F| for that
// component.  With VEC the accumulator rows are padded to 4-aligned x groups
// of the field ([ox-4, ox+2^l+4)) and flushed with 16-byte vector atomics
// (zero lanes of a group add nothing).  A chunk with non-finite forces is
// added directly.
template <typename FT, bool VEC, int LX, int LY = 0, int LZ = 0>
__global__ void __launch_bounds__(kSpreadThreads, 8) k_spread(Dims D, Tiles tl, const float* __restrict__ phi,
                                                           const float* __restrict__ cl,
                                                           const int32_t* __restrict__ home,
                                                           const int32_t* __restrict__ perm,
                                                           const int32_t* __restrict__ items,
                                                           const int32_t* __restrict__ n_items_p,
                                                           const int32_t* __restrict__ offsets,
                                                           const int32_t* __restrict__ counts, int64_t M, int64_t cap,
                                                           const float* __restrict__ F, FT* __restrict__ f) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int XOFF = VEC ? 4 : 1;
  constexpr int AX = (1 << LX) + 2 * XOFF;
  const int ly = LY ? LY : tl.l[1], lz = LZ ? LZ : tl.l[2];   // compile-time when specialised
  const AccShape A(LX, ly, lz, VEC);
  const SpreadSmem L(4, LX, ly, lz, VEC);
  const int AY = A.AY, PS = A.PS, ACC = A.ACC, ROWS = AY * A.AZ;
  int* acc = reinterpret_cast<int*>(smem_raw);
  int* row_a = reinterpret_cast<int*>(smem_raw + L.rows);
  int* row_g = row_a + ROWS;
  unsigned char* flag = reinterpret_cast<unsigned char*>(row_g + ROWS);
  __shared__ float s_red[3 * (kSpreadThreads / 32)];
  const int tid = threadIdx.x;
  const int64_t N = (int64_t)D.n[0] * D.n[1] * D.n[2];
  const int n_items = *n_items_p;
  for (int e = tid; e < 3 * ACC; e += kSpreadThreads) acc[e] = 0;
  for (int r = tid; r < ROWS; r += kSpreadThreads) flag[r] = 0;

  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int b = items[it];
    const int start = offsets[b], cnt = counts[b];
    const int bx = b % tl.nb[0], by = (b / tl.nb[0]) % tl.nb[1], bz = b / (tl.nb[0] * tl.nb[1]);
    const int ox = bx << LX, oy = by << ly, oz = bz << lz;
    for (int r = tid; r < ROWS; r += kSpreadThreads) {
      const int ey = r % AY, ez = r / AY;
      row_a[r] = ez * PS + ey * AX;
      row_g[r] = wrap(oz - 1 + ez, D.n[2], D.periodic[2]) * D.n[1] + wrap(oy - 1 + ey, D.n[1], D.periodic[1]);
    }
    for (int j0 = start; j0 < start + cnt; j0 += kSpreadThreads) {
      const int64_t j = j0 + tid;
      const bool act = j < start + cnt;
      int i[3] = {0, 0, 0};
      float v[3] = {0.f, 0.f, 0.f};
      // The marker's 27 phi values are loaded before the chunk's barrier, so
      // their latency overlaps the block-wide maximum.
      float p[27];
#pragma unroll
      for (int k = 0; k < 27; ++k) p[k] = 0.f;
      if (act) {
#pragma unroll
        for (int k = 0; k < 27; ++k) p[k] = phi[k * cap + j];
        decode_home(home[j], D, i);
        const int64_t m = perm[j];
        const float c = cl[j];
        v[0] = c * F[m];
        v[1] = c * F[M + m];
        v[2] = c * F[2 * M + m];
      }
      float vm[3] = {fabsf(v[0]), fabsf(v[1]), fabsf(v[2])};
      block_max3(vm, s_red);                         // barrier inside: row tables and resets are complete
      const float vmax = fmaxf(vm[0], fmaxf(vm[1], vm[2]));
      if (vmax == 0.f) {
        __syncthreads();
        continue;
      }
      if (!isfinite(vmax)) {
        if (act) {
          for (int k = 0; k < 27; ++k) {
            const int gx = wrap(i[0] + k % 3 - 1, D.n[0], D.periodic[0]);
            const int gy = wrap(i[1] + (k / 3) % 3 - 1, D.n[1], D.periodic[1]);
            const int gz = wrap(i[2] + k / 9 - 1, D.n[2], D.periodic[2]);
            const int64_t o = ((int64_t)gz * D.n[1] + gy) * D.n[0] + gx;
            const float p = phi[k * cap + j];
            for (int q = 0; q < 3; ++q) add_field<float, FT>(f + q * N + o, p * v[q]);
          }
        }
        __syncthreads();
        continue;
      }
      // Per component: vm < 2^ex, scale 2^(23 - ex) keeps |p v| * scale <= 2^22 for |p| <= 1/2.
      float scale[3], inv_scale[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        int ex;
        frexpf(vm[q] > 0.f ? vm[q] : vmax, &ex);
        scale[q] = ldexpf(1.f, 23 - ex);
        inv_scale[q] = ldexpf(1.f, ex - 23);
      }
      if (act) {
        const float q0 = v[0] * scale[0], q1 = v[1] * scale[1], q2 = v[2] * scale[2];
        const int lx = i[0] - ox, ly = i[1] - oy, lz = i[2] - oz;
        const int base = lz * PS + ly * AX + lx + XOFF - 1;
        const int r0 = lz * AY + ly;
#pragma unroll
        for (int cz = 0; cz < 3; ++cz)
#pragma unroll
          for (int cy = 0; cy < 3; ++cy) flag[r0 + cz * AY + cy] = 1;
        float pmax = 0.f;
#pragma unroll
        for (int k = 0; k < 27; ++k) pmax = fmaxf(pmax, fabsf(p[k]));
        if (pmax <= 0.5f) {
          add_stencil_fixed(acc + base, p, q0, q1, q2, PS, AX, ACC);
        } else {
#pragma unroll
          for (int k = 0; k < 27; ++k) {
            const int li = base + (k / 9) * PS + ((k / 3) % 3) * AX + k % 3;
            if (fabsf(p[k]) <= 0.5f) {
              atomicAdd(&acc[li], round_mul(p[k], q0));
              atomicAdd(&acc[ACC + li], round_mul(p[k], q1));
              atomicAdd(&acc[2 * ACC + li], round_mul(p[k], q2));
            } else {
              const int gx = wrap(i[0] + k % 3 - 1, D.n[0], D.periodic[0]);
              const int gy = wrap(i[1] + (k / 3) % 3 - 1, D.n[1], D.periodic[1]);
              const int gz = wrap(i[2] + k / 9 - 1, D.n[2], D.periodic[2]);
              const int64_t o = ((int64_t)gz * D.n[1] + gy) * D.n[0] + gx;
              add_field<float, FT>(f + o, p[k] * v[0]);
              add_field<float, FT>(f + N + o, p[k] * v[1]);
              add_field<float, FT>(f + 2 * N + o, p[k] * v[2]);
            }
          }
        }
      }
      __syncthreads();
      if (VEC) {
        constexpr int G = AX / 4;
        for (int g = tid; g < G * ROWS; g += kSpreadThreads) {
          const int row = g / G, q = g - row * G;
          if (!flag[row]) continue;
          const int e = row_a[row] + 4 * q;
          int4* p0 = reinterpret_cast<int4*>(&acc[e]);
          int4* p1 = reinterpret_cast<int4*>(&acc[ACC + e]);
          int4* p2 = reinterpret_cast<int4*>(&acc[2 * ACC + e]);
          const int4 a0 = *p0, a1 = *p1, a2 = *p2;
          const bool n0 = (a0.x | a0.y | a0.z | a0.w) != 0;
          const bool n1 = (a1.x | a1.y | a1.z | a1.w) != 0;
          const bool n2 = (a2.x | a2.y | a2.z | a2.w) != 0;
          if (!(n0 || n1 || n2)) continue;
          const int4 z = make_int4(0, 0, 0, 0);
          *p0 = z;
          *p1 = z;
          *p2 = z;
          int gx = ox - XOFF + 4 * q;
          if (gx < 0 || gx >= D.n[0]) {
            if (!D.periodic[0]) continue;
            gx = gx < 0 ? gx + D.n[0] : gx - D.n[0];
            if (gx < 0 || gx >= D.n[0]) continue;        // padding beyond one period holds no sums
          }
          FT* fo = f + (int64_t)row_g[row] * D.n[0] + gx;
          const float u0 = inv_scale[0], u1 = inv_scale[1], u2 = inv_scale[2];
          if (n0) red_add_v4(fo, a0.x * u0, a0.y * u0, a0.z * u0, a0.w * u0);
          if (n1) red_add_v4(fo + N, a1.x * u1, a1.y * u1, a1.z * u1, a1.w * u1);
          if (n2) red_add_v4(fo + 2 * N, a2.x * u2, a2.y * u2, a2.z * u2, a2.w * u2);
        }
      } else {
        for (int e = tid; e < AX * ROWS; e += kSpreadThreads) {
          const int row = e / AX, ex = e - row * AX;
          if (!flag[row]) continue;
          const int li = row_a[row] + ex;
          const int a0 = acc[li], a1 = acc[ACC + li], a2 = acc[2 * ACC + li];
          if ((a0 | a1 | a2) == 0) continue;
          acc[li] = 0;
          acc[ACC + li] = 0;
          acc[2 * ACC + li] = 0;
          const int gx = wrap(ox - XOFF + ex, D.n[0], D.periodic[0]);
          const int64_t o = (int64_t)row_g[row] * D.n[0] + gx;
          if (a0) add_field<float, FT>(f + o, a0 * inv_scale[0]);
          if (a1) add_field<float, FT>(f + N + o, a1 * inv_scale[1]);
          if (a2) add_field<float, FT>(f + 2 * N + o, a2 * inv_scale[2]);
        }
      }
      __syncthreads();
      for (int r = tid; r < ROWS; r += kSpreadThreads) flag[r] = 0;
    }
  }
}

// Double-precision spreading (the small double-precision workloads): one
// thread per stored marker adds its 27 x 3 terms c_l phi_k F_l straight into
// f with native global double reductions.  Shared-memory accumulation, as in
// single precision, needs double shared atomics, which are compare-and-swap
// loops on this GPU and serialise badly where markers crowd few cells.
__global__ void __launch_bounds__(kBlock) k_spread_f64(Dims D, const double* __restrict__ phi,
                                                       const double* __restrict__ cl, const int32_t* __restrict__ home,
                                                       const int32_t* __restrict__ perm, int64_t M, int64_t cap,
                                                       const double* __restrict__ F, double* __restrict__ f) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const int32_t h = home[j];
  if (h < 0) return;
  int i[3];
  decode_home(h, D, i);
  const int64_t m = perm[j];
  const double c = cl[j];
  const double v0 = c * F[m], v1 = c * F[M + m], v2 = c * F[2 * M + m];
  const int64_t N = (int64_t)D.n[0] * D.n[1] * D.n[2];
#pragma unroll
  for (int cz = 0; cz < 3; ++cz) {
    const int gz = wrap(i[2] + cz - 1, D.n[2], D.periodic[2]);
#pragma unroll
    for (int cy = 0; cy < 3; ++cy) {
      const int64_t row = ((int64_t)gz * D.n[1] + wrap(i[1] + cy - 1, D.n[1], D.periodic[1])) * D.n[0];
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) {
        const double p = phi[(9 * cz + 3 * cy + cx) * cap + j];
        const int64_t o = row + wrap(i[0] + cx - 1, D.n[0], D.periodic[0]);
        atomicAdd(f + o, p * v0);
        atomicAdd(f + N + o, p * v1);
        atomicAdd(f + 2 * N + o, p * v2);
      }
    }
  }
}

size_t spread_smem_bytes(const mls_ctx* ctx) {
  if (ctx->opt.real == MLS_F64) return 0;   // the double-precision spread uses no shared memory
  return (size_t)SpreadSmem(4, ctx->tiles.l[0], ctx->tiles.l[1], ctx->tiles.l[2], spread_vec(ctx)).total;
}

template <typename K>
static cudaError_t configure_kernel(mls_ctx* ctx, K kernel, int smem) {
  cudaError_t e = raise_smem_limit((const void*)kernel, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0, dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kSpreadThreads, smem);
  if (e != cudaSuccess) return e;
  ctx->spread_grid = (per_sm > 0 ? per_sm : 1) * sms;
  ctx->spread_threads = kSpreadThreads;
  return cudaSuccess;
}

template <typename FT, bool VEC>
static const void* spread_kernel(int lx, int ly, int lz) {
  // Tile shapes the tile-shape tuner tries get compile-time accumulator strides.
  if (VEC) {
    if (lx == 3 && ly == 3 && lz == 3) return (const void*)k_spread<FT, VEC, 3, 3, 3>;
    if (lx == 3 && ly == 3 && lz == 2) return (const void*)k_spread<FT, VEC, 3, 3, 2>;
    if (lx == 4 && ly == 3 && lz == 3) return (const void*)k_spread<FT, VEC, 4, 3, 3>;
    if (lx == 4 && ly == 4 && lz == 3) return (const void*)k_spread<FT, VEC, 4, 4, 3>;
    if (lx == 4 && ly == 4 && lz == 2) return (const void*)k_spread<FT, VEC, 4, 4, 2>;
    if (lx == 5 && ly == 3 && lz == 3) return (const void*)k_spread<FT, VEC, 5, 3, 3>;
  }
  switch (lx) {
    case 1: return VEC ? nullptr : (const void*)k_spread<FT, false, 1>;
    case 2: return (const void*)k_spread<FT, VEC, 2>;
    case 3: return (const void*)k_spread<FT, VEC, 3>;
    case 4: return (const void*)k_spread<FT, VEC, 4>;
    default: return (const void*)k_spread<FT, VEC, 5>;
  }
}

static cudaError_t interp_configure(mls_ctx* ctx) {
  if (ctx->opt.real == MLS_F64) return cudaSuccess;
  const int smem = InterpSmem(ctx->tiles.l[0], ctx->tiles.l[1], ctx->tiles.l[2], ctx->opt.field == MLS_BF16).total;
  const void* k = ctx->opt.field == MLS_F32 ? interp_kernel<float>(ctx->tiles.l[0])
                                            : interp_kernel<__nv_bfloat16>(ctx->tiles.l[0]);
  cudaError_t e;
  if ((e = raise_smem_limit(k, smem)) != cudaSuccess) return e;
  int per_sm = 0, sms = 0, dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kInterpThreads, smem)) != cudaSuccess) return e;
  ctx->interp_grid = (per_sm > 0 ? per_sm : 1) * sms;
  return cudaSuccess;
}

cudaError_t spread_configure(mls_ctx* ctx) {
  const cudaError_t ei = interp_configure(ctx);
  if (ei != cudaSuccess) return ei;
  const int smem = (int)spread_smem_bytes(ctx);
  const int lx = ctx->tiles.l[0], ly = ctx->tiles.l[1], lz = ctx->tiles.l[2];
  if (ctx->opt.real == MLS_F64) return cudaSuccess;
  const bool bf = ctx->opt.field == MLS_BF16;
  if (spread_vec(ctx)) {
    // The scalar variant also runs when f is not aligned for the vector reductions (same layout size or smaller).
    cudaError_t e = configure_kernel(ctx, bf ? spread_kernel<__nv_bfloat16, false>(lx, ly, lz) : spread_kernel<float, false>(lx, ly, lz),
                                     smem);
    if (e != cudaSuccess) return e;
    return configure_kernel(ctx, bf ? spread_kernel<__nv_bfloat16, true>(lx, ly, lz) : spread_kernel<float, true>(lx, ly, lz), smem);
  }
  return configure_kernel(ctx, bf ? spread_kernel<__nv_bfloat16, false>(lx, ly, lz) : spread_kernel<float, false>(lx, ly, lz), smem);
}

cudaError_t launch_interp(const mls_ctx* ctx, const mls_transfer* T, const void* u, void* U, cudaStream_t s) {
  if (T->M == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((T->M + kBlock - 1) / kBlock);
  const Dims D = dims_of(ctx);
  if (ctx->opt.real == MLS_F64)
    k_interp<double, double><<<grid, kBlock, 0, s>>>(D, (const double*)T->phi, T->home, T->perm, T->M, T->cap,
                                                     (const double*)u, (double*)U);
  else {
    Tiles tl = ctx->tiles;
    const float* phi = (const float*)T->phi;
    int64_t M = T->M, cap = T->cap;
    const bool bf = ctx->opt.field == MLS_BF16;
    int pairs = bf && D.n[0] % 2 == 0 && (reinterpret_cast<uintptr_t>(u) & 3) == 0 ? 1 : 0;
    void* args[] = {(void*)&D, &tl, (void*)&phi, (void*)&T->home, (void*)&T->perm, (void*)&T->items,
                    (void*)&T->n_items, (void*)&T->offsets, (void*)&T->counts, &M, &cap, (void*)&u, &U, &pairs};
    const void* k = bf ? interp_kernel<__nv_bfloat16>(tl.l[0]) : interp_kernel<float>(tl.l[0]);
    return cudaLaunchKernel(k, dim3(ctx->interp_grid), dim3(kInterpThreads), args,
                            (size_t)InterpSmem(tl.l[0], tl.l[1], tl.l[2], bf).total, s);
  }
  return cudaGetLastError();
}

template <typename FT, bool VEC>
static cudaError_t launch_spread_one(const mls_ctx* ctx, const mls_transfer* T, const void* F, void* f,
                                     cudaStream_t s) {
  Dims D = dims_of(ctx);
  Tiles tl = ctx->tiles;
  const float* phi = (const float*)T->phi;
  const float* c = (const float*)T->c;
  int64_t M = T->M, cap = T->cap;
  void* args[] = {&D, &tl, (void*)&phi, (void*)&c, (void*)&T->home, (void*)&T->perm, (void*)&T->items,
                  (void*)&T->n_items, (void*)&T->offsets, (void*)&T->counts, &M, &cap, (void*)&F, &f};
  return cudaLaunchKernel(spread_kernel<FT, VEC>(tl.l[0], tl.l[1], tl.l[2]), dim3(ctx->spread_grid), dim3(ctx->spread_threads), args,
                          spread_smem_bytes(ctx), s);
}

cudaError_t launch_spread(const mls_ctx* ctx, const mls_transfer* T, const void* F, void* f, cudaStream_t s) {
  if (T->M == 0) return cudaSuccess;
  if (ctx->opt.real == MLS_F64)
    k_spread_f64<<<(unsigned)((T->M + kBlock - 1) / kBlock), kBlock, 0, s>>>(
        dims_of(ctx), (const double*)T->phi, (const double*)T->c, T->home, T->perm, T->M, T->cap,
        (const double*)F, (double*)f);
  else if (ctx->opt.field == MLS_BF16)
    return spread_vec_aligned(ctx, f) ? launch_spread_one<__nv_bfloat16, true>(ctx, T, F, f, s)
                                      : launch_spread_one<__nv_bfloat16, false>(ctx, T, F, f, s);
  else if (spread_vec_aligned(ctx, f))
    return launch_spread_one<float, true>(ctx, T, F, f, s);
  else return launch_spread_one<float, false>(ctx, T, F, f, s);
  return cudaGetLastError();
}

}  // namespace mls
