// The fused direct-forcing kernel (interpolation, the IBM force and spreading
// in one pass over the spreading tiles, reading phi once) and its instance
// selector, shared by the translation units that instantiate it for each
// block size.
#pragma once

#include "transfer_common.cuh"

namespace mls {

// Shared memory of one fused block: the spreading accumulator (3 components,
// AccShape), the field brick (3 components, InterpSmem geometry: rows of
// 2^lx + 2 cells), then per tile row (y, z) its accumulator offset, its brick
// offset, its global row index and a touched flag.  Both geometries have
// the same (2^ly + 2) x (2^lz + 2) rows.
struct ForceSmem {
  int brick, rows, total;
  __host__ __device__ ForceSmem(int lx, int ly, int lz, bool vec) {
    const AccShape A(lx, ly, lz, vec);
    const InterpSmem B(lx, ly, lz);
    const int R = A.AY * A.AZ;
    brick = (3 * A.ACC * 4 + 15) & ~15;
    rows = (brick + 3 * B.CELLS * 4 + 15) & ~15;
    total = (rows + 12 * R + R + 15) & ~15;
  }
};

// Direct forcing (Section 2, text after Eq. 6 and Eq. 7), single precision:
// U_l = sum_k phi_k^l u_k, F_l = (V_b,l - U_l) / dt, f_k += sum_l c_l phi_k^l F_l.
// Persistent blocks walk the non-empty spreading tiles.  For a tile, every
// marker flags the 9 rows (y, z) its support touches; the flagged rows of u
// are copied into a shared-memory brick; then per chunk of up to NT (the
// block size: 256 or 128) markers each thread loads its marker's 27 phi once,
// gathers U from the brick, forms F (written to F and, if requested, U in
// caller order) and adds c phi F into the int32 fixed-point accumulator as
// k_spread does (per-component power-of-two scale per chunk, so that a cell
// sum stays below 256 * 2^22 = 2^30; |phi| > 1/2 terms and non-finite chunks
// added directly); the flagged rows are flushed with vector reductions (VEC)
// or scalar atomics and reset.  Markers without support (the last bin of the
// tile sort) get U = F = 0.
template <typename FT, bool VEC, int LX, int LY, int LZ, int NT>
__global__ void __launch_bounds__(NT) k_direct_forcing(
    Dims D, Tiles tl, const float* __restrict__ phi, const float* __restrict__ cl, const int32_t* __restrict__ home,
    const int32_t* __restrict__ perm, const int32_t* __restrict__ items, const int32_t* __restrict__ n_items_p,
    const int32_t* __restrict__ offsets, const int32_t* __restrict__ counts, int64_t M, int64_t cap,
    const FT* __restrict__ u, const float* __restrict__ Vb, float inv_dt, float* __restrict__ U,
    float* __restrict__ Fout, FT* __restrict__ f) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int XOFF = VEC ? 4 : 1;
  constexpr int AX = (1 << LX) + 2 * XOFF;
  constexpr int BX = (1 << LX) + 2;
  const int ly = LY ? LY : tl.l[1], lz = LZ ? LZ : tl.l[2];   // compile-time when specialised
  const AccShape A(LX, ly, lz, VEC);
  const InterpSmem B(LX, ly, lz);
  const ForceSmem L(LX, ly, lz, VEC);
  const int AY = A.AY, PS = A.PS, ACC = A.ACC, ROWS = AY * A.AZ;
  const int BPS = B.PS, CELLS = B.CELLS;
  int* acc = reinterpret_cast<int*>(smem_raw);
  float* su = reinterpret_cast<float*>(smem_raw + L.brick);
  int* row_a = reinterpret_cast<int*>(smem_raw + L.rows);
  int* row_s = row_a + ROWS;
  int* row_g = row_s + ROWS;
  unsigned char* flag = reinterpret_cast<unsigned char*>(row_g + ROWS);
  __shared__ float s_red[3 * (NT / 32)];
  const int tid = threadIdx.x;
  const int64_t N = (int64_t)D.n[0] * D.n[1] * D.n[2];
  const int n_items = *n_items_p;
  for (int e = tid; e < 3 * ACC; e += NT) acc[e] = 0;
  for (int r = tid; r < ROWS; r += NT) flag[r] = 0;
  __syncthreads();

  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int b = items[it];
    const int start = offsets[b], end = start + counts[b];
    const int bx = b % tl.nb[0], by = (b / tl.nb[0]) % tl.nb[1], bz = b / (tl.nb[0] * tl.nb[1]);
    const int ox = bx << LX, oy = by << ly, oz = bz << lz;
    // Touched rows of the whole tile (plain byte stores) and the row tables.
    for (int j = start + tid; j < end; j += NT) {
      int i[3];
      decode_home(home[j], D, i);
      const int r0 = (i[2] - oz) * AY + (i[1] - oy);
#pragma unroll
      for (int cz = 0; cz < 3; ++cz)
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) flag[r0 + cz * AY + cy] = 1;
    }
    for (int r = tid; r < ROWS; r += NT) {
      const int ey = r % AY, ez = r / AY;
      row_a[r] = ez * PS + ey * AX;
      row_s[r] = ez * BPS + ey * BX;
      row_g[r] = wrap(oz - 1 + ez, D.n[2], D.periodic[2]) * D.n[1] + wrap(oy - 1 + ey, D.n[1], D.periodic[1]);
    }
    __syncthreads();
    // The touched rows of u into the brick.
    for (int e = tid; e < ROWS * BX; e += NT) {
      const int r = e / BX, ex = e - r * BX;
      if (!flag[r]) continue;
      const int gx = wrap(ox - 1 + ex, D.n[0], D.periodic[0]);
      stage_cell(su + row_s[r] + ex, CELLS, u, N, (int64_t)row_g[r] * D.n[0] + gx);
    }
    cp_async_wait_all();
    __syncthreads();

    for (int j0 = start; j0 < end; j0 += NT) {
      const int64_t j = j0 + tid;
      const bool act = j < end;
      int i[3] = {0, 0, 0};
      float v[3] = {0.f, 0.f, 0.f};
      float p[27];
      if (act) {
        decode_home(home[j], D, i);
        const int64_t m = perm[j];
        const float c = cl[j];
#pragma unroll
        for (int k = 0; k < 27; ++k) p[k] = phi[k * cap + j];
        const int base = (i[2] - oz) * BPS + (i[1] - oy) * BX + (i[0] - ox);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int cz = 0; cz < 3; ++cz)
#pragma unroll
          for (int cy = 0; cy < 3; ++cy)
#pragma unroll
            for (int cx = 0; cx < 3; ++cx) {
              const float pk = p[9 * cz + 3 * cy + cx];
              const int si = base + cz * BPS + cy * BX + cx;
              s0 += pk * su[si];
              s1 += pk * su[CELLS + si];
              s2 += pk * su[2 * CELLS + si];
            }
        const float F0 = (Vb[m] - s0) * inv_dt, F1 = (Vb[M + m] - s1) * inv_dt, F2 = (Vb[2 * M + m] - s2) * inv_dt;
        if (U) {
          U[m] = s0;
          U[M + m] = s1;
          U[2 * M + m] = s2;
        }
        Fout[m] = F0;
        Fout[M + m] = F1;
        Fout[2 * M + m] = F2;
        v[0] = c * F0;
        v[1] = c * F1;
        v[2] = c * F2;
      }
      float vm[3] = {fabsf(v[0]), fabsf(v[1]), fabsf(v[2])};
      block_max3<NT>(vm, s_red);
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
            for (int q = 0; q < 3; ++q) add_field<float, FT>(f + q * N + o, p[k] * v[q]);
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
        const int base = (i[2] - oz) * PS + (i[1] - oy) * AX + (i[0] - ox) + XOFF - 1;
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
        for (int g = tid; g < G * ROWS; g += NT) {
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
        for (int e = tid; e < AX * ROWS; e += NT) {
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
    }
    // The tile's flags are cleared once all its chunks are flushed; the next
    // tile sets its own only after the barrier.
    for (int r = tid; r < ROWS; r += NT) flag[r] = 0;
    __syncthreads();
  }
  // Markers without support: no interpolated velocity and no force.
  const int64_t d0 = offsets[tl.nbins - 1];
  for (int64_t j = d0 + (int64_t)blockIdx.x * NT + tid; j < M;
       j += (int64_t)gridDim.x * NT) {
    const int64_t m = perm[j];
    if (U) {
      U[m] = 0.f;
      U[M + m] = 0.f;
      U[2 * M + m] = 0.f;
    }
    Fout[m] = 0.f;
    Fout[M + m] = 0.f;
    Fout[2 * M + m] = 0.f;
  }
}

template <typename FT, bool VEC, int NT>
inline const void* force_kernel(int lx, int ly, int lz) {
  // Tile shapes the tile-shape tuner tries get compile-time strides.
  if (VEC) {
    if (lx == 3 && ly == 3 && lz == 3) return (const void*)k_direct_forcing<FT, VEC, 3, 3, 3, NT>;
    if (lx == 3 && ly == 3 && lz == 2) return (const void*)k_direct_forcing<FT, VEC, 3, 3, 2, NT>;
    if (lx == 4 && ly == 3 && lz == 3) return (const void*)k_direct_forcing<FT, VEC, 4, 3, 3, NT>;
    if (lx == 4 && ly == 4 && lz == 3) return (const void*)k_direct_forcing<FT, VEC, 4, 4, 3, NT>;
    if (lx == 4 && ly == 4 && lz == 2) return (const void*)k_direct_forcing<FT, VEC, 4, 4, 2, NT>;
    if (lx == 5 && ly == 3 && lz == 3) return (const void*)k_direct_forcing<FT, VEC, 5, 3, 3, NT>;
  }
  switch (lx) {
    case 1: return VEC ? nullptr : (const void*)k_direct_forcing<FT, false, 1, 0, 0, NT>;
    case 2: return (const void*)k_direct_forcing<FT, VEC, 2, 0, 0, NT>;
    case 3: return (const void*)k_direct_forcing<FT, VEC, 3, 0, 0, NT>;
    case 4: return (const void*)k_direct_forcing<FT, VEC, 4, 0, 0, NT>;
    default: return (const void*)k_direct_forcing<FT, VEC, 5, 0, 0, NT>;
  }
}

// The instance for a context's tile shape and field type, for blocks of 256
// threads (k_force_256.cu) and of 128 (k_force.cu).
const void* force_kernel_256(bool bf, bool vec, int lx, int ly, int lz);
const void* force_kernel_128(bool bf, bool vec, int lx, int ly, int lz);

}  // namespace mls
