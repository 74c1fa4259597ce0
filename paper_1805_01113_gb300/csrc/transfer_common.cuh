// Device helpers shared by the transfer kernels (interpolation, spreading,
// the fused direct-forcing step): grid dimensions and home-cell decoding,
// shared-memory brick and accumulator geometry, asynchronous copies, vector
// reductions and the fixed-point rounding of the spreading accumulators.
#pragma once

#include "mls_host.h"

namespace mls {

template <typename FT> __device__ __forceinline__ float to_f(FT v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename R, typename FT> __device__ __forceinline__ R load_field(const FT* p) {
  return (R)to_f<FT>(__ldg(p));
}
template <> __device__ __forceinline__ double load_field<double, double>(const double* p) { return __ldg(p); }

// Division by a fixed divisor d >= 1 of numerators n < 2^31 by one 64-bit
// multiply: with l = ceil(log2 d) and m = floor(2^(32+l) / d) + 1, the error
// of m / 2^(32+l) against 1/d is below 1 / (d 2^(32+l)) per unit of n, so
// floor(n m / 2^(32+l)) = floor(n / d) while n < 2^31 <= 2^(32+l) / 2.
struct FastDiv {
  unsigned long long m;
  int shift;
  int d;
  void init(int divisor) {
    d = divisor;
    int l = 0;
    while ((1LL << l) < (long long)divisor) ++l;
    shift = 32 + l;
    m = (unsigned long long)(((unsigned __int128)1 << shift) / (unsigned)divisor) + 1ULL;
  }
  __device__ __forceinline__ int div(int n) const { return (int)(((unsigned long long)(unsigned)n * m) >> shift); }
};

struct Dims {
  int n[3];
  int periodic[3];
  FastDiv div0, div1;  // by n[0] and by n[1]
};

__device__ __forceinline__ void decode_home(int32_t h, const Dims& D, int i[3]) {
  const int r = D.div0.div(h);
  i[0] = h - r * D.n[0];
  i[2] = D.div1.div(r);
  i[1] = r - i[2] * D.n[1];
}

// Asynchronous 4-byte global-to-shared copy (no register round trip).
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void stage_cell(float* dst, int stride, const float* u, int64_t N, int64_t o) {
  cp_async4(dst, u + o);
  cp_async4(dst + stride, u + N + o);
  cp_async4(dst + 2 * stride, u + 2 * N + o);
}
__device__ __forceinline__ void stage_cell(float* dst, int stride, const __nv_bfloat16* u, int64_t N, int64_t o) {
  const float v0 = __bfloat162float(u[o]), v1 = __bfloat162float(u[N + o]), v2 = __bfloat162float(u[2 * N + o]);
  dst[0] = v0;
  dst[stride] = v1;
  dst[2 * stride] = v2;
}

// Field brick of a spreading tile for interpolation: the tile plus a
// one-cell halo, rows of BX = 2^lx + 2 cells, BY rows per plane, BZ planes of
// stride PS (padded by 4 cells against bank aliasing), three components;
// then per brick row its offset in the brick, its global row index and a
// touched flag.  A bfloat16 brick keeps the field's 2-byte values and starts
// each row one cell further left (rows of 2^lx + 4 cells, [ox - 2, ox + 2^lx + 2)),
// so that it is copied in 4-byte pairs that start on even cells.
struct InterpSmem {
  int BX, BY, BZ, PS, CELLS, ROWS, rows, total;
  __host__ __device__ InterpSmem(int lx, int ly, int lz, bool bf16 = false) {
    BX = (1 << lx) + (bf16 ? 4 : 2);
    BY = (1 << ly) + 2;
    BZ = (1 << lz) + 2;
    PS = BY * BX + 4;
    CELLS = BZ * PS;
    ROWS = BY * BZ;
    rows = (3 * CELLS * (bf16 ? 2 : 4) + 15) & ~15;
    total = (rows + 8 * ROWS + ROWS + 15) & ~15;
  }
};

// Asynchronous 4-byte copy of a pair of bfloat16 values.
__device__ __forceinline__ void cp_async4_pair(__nv_bfloat16* dst, const __nv_bfloat16* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}

// Adds four consecutive cells of a field with one vector reduction:
// 16 bytes of float, or 8 bytes (two bf16x2 pairs) of bfloat16.
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}
__device__ __forceinline__ void red_add_v4(__nv_bfloat16* p, float a, float b, float c, float d) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  asm volatile("red.global.add.noftz.v2.bf16x2 [%0], {%1, %2};" ::"l"(p),
               "r"(*reinterpret_cast<const unsigned*>(&lo)), "r"(*reinterpret_cast<const unsigned*>(&hi))
               : "memory");
}

template <typename R, typename FT> __device__ __forceinline__ void add_field(FT* p, R v);
template <> __device__ __forceinline__ void add_field<double, double>(double* p, double v) { atomicAdd(p, v); }
template <> __device__ __forceinline__ void add_field<float, float>(float* p, float v) { atomicAdd(p, v); }
template <> __device__ __forceinline__ void add_field<float, __nv_bfloat16>(__nv_bfloat16* p, float v) {
  atomicAdd(p, __float2bfloat16_rn(v));
}

// Accumulator geometry of a spreading tile (tile plus one-cell halo): rows
// of AX cells (x padded to 4-aligned field groups with VEC), AY rows per
// plane, AZ planes.  Planes are padded by 4 cells so that cells of one
// column in different planes fall in different shared-memory banks (with a
// plane of a multiple of 32 cells every plane would alias the same banks).
struct AccShape {
  int AX, AY, AZ, PS, ACC, XOFF;
  __host__ __device__ AccShape(int lx, int ly, int lz, bool vec) {
    XOFF = vec ? 4 : 1;
    AX = (1 << lx) + 2 * XOFF;
    AY = (1 << ly) + 2;
    AZ = (1 << lz) + 2;
    PS = AY * AX + 4;
    ACC = AZ * PS;
  }
};

// Shared-memory bytes of one spreading block: the accumulator (3 components),
// then per accumulator row (y, z) its offset in the accumulator, its global
// row index and a touched flag.
struct SpreadSmem {
  int rows, total;
  __host__ __device__ SpreadSmem(int rs, int lx, int ly, int lz, bool vec) {
    const AccShape A(lx, ly, lz, vec);
    const int R = A.AY * A.AZ;
    rows = (3 * A.ACC * rs + 15) & ~15;
    total = (rows + 8 * R + R + 15) & ~15;
  }
};

template <int NT = kSpreadThreads>
__device__ __forceinline__ void block_max3(float v[3], float* red) {
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] = fmaxf(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[3 * w] = v[0];
    red[3 * w + 1] = v[1];
    red[3 * w + 2] = v[2];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    float m = red[q];
    for (int ww = 1; ww < NT / 32; ++ww) m = fmaxf(m, red[3 * ww + q]);
    v[q] = m;
  }
}

// round-to-nearest integer of a * b for |a b| <= 2^22, in one fused
// multiply-add: a b + 1.5 * 2^23 lies in [2^23, 2^24), where the float spacing
// is 1, so the single rounding of the fma leaves round(a b) in the low
// mantissa bits.
__device__ __forceinline__ int round_mul(float a, float b) {
  return __float_as_int(__fmaf_rn(a, b, 12582912.0f)) - 0x4B400000;
}

// Adds one marker's 27 x 3 fixed-point terms round(phi_k q_c) into the shared
// accumulator, a0 pointing at the stencil's (-1,-1,-1) cell, rows AX cells
// apart, planes PS, components ACC.  Markers of one warp often share a home
// cell (inside a tile, markers are ordered by home cell), and lanes that add
// to one word in the same instruction are serialised.  So each lane walks the
// stencil in its own order: x rotated by lane % 3 and z by (lane / 3) % 3;
// at step (cz, cy, cx) the lane adds node ((cz + rc) % 3, cy, (cx + ra) % 3).
// The integer sums do not depend on the order.
// Picks a (r == 0), b (r == 1) or c (r == 2) with two predicated selects,
// so that the rotation below stays branch-free (lanes differ in r).
__device__ __forceinline__ float select3(int r, float a, float b, float c) {
  float bc, o;
  asm("{\n\t.reg .pred q;\n\tsetp.eq.s32 q, %1, 1;\n\tselp.f32 %0, %2, %3, q;\n\t}" : "=f"(bc) : "r"(r), "f"(b), "f"(c));
  asm("{\n\t.reg .pred q;\n\tsetp.eq.s32 q, %1, 0;\n\tselp.f32 %0, %2, %3, q;\n\t}" : "=f"(o) : "r"(r), "f"(a), "f"(bc));
  return o;
}

__device__ __forceinline__ void add_stencil_fixed(int* a0, const float p[27], float q0, float q1, float q2, int PS,
                                                  int AX, int ACC) {
  const int lane = threadIdx.x & 31;
  const int ra = lane % 3, rc = (lane / 3) % 3;
  float t[27];
#pragma unroll
  for (int r = 0; r < 9; ++r) {
    const float v0 = p[3 * r], v1 = p[3 * r + 1], v2 = p[3 * r + 2];
    t[3 * r] = select3(ra, v0, v1, v2);
    t[3 * r + 1] = select3(ra, v1, v2, v0);
    t[3 * r + 2] = select3(ra, v2, v0, v1);
  }
  const int xo[3] = {ra, ra == 2 ? 0 : ra + 1, ra == 0 ? 2 : ra - 1};
  const int zo[3] = {rc * PS, (rc == 2 ? 0 : rc + 1) * PS, (rc == 0 ? 2 : rc - 1) * PS};
#pragma unroll
  for (int cz = 0; cz < 3; ++cz) {
    const int z1 = (cz + 1) % 3, z2 = (cz + 2) % 3;
#pragma unroll
    for (int cy = 0; cy < 3; ++cy) {
      int* ar = a0 + zo[cz] + cy * AX;
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) {
        const int m = 3 * cy + cx;
        const float pk = select3(rc, t[9 * cz + m], t[9 * z1 + m], t[9 * z2 + m]);
        int* a = ar + xo[cx];
        atomicAdd(a, round_mul(pk, q0));
        atomicAdd(a + ACC, round_mul(pk, q1));
        atomicAdd(a + 2 * ACC, round_mul(pk, q2));
      }
    }
  }
}

inline Dims dims_of(const mls_ctx* ctx) {
  Dims D;
  for (int d = 0; d < 3; ++d) {
    D.n[d] = ctx->n[d];
    D.periodic[d] = ctx->periodic[d];
  }
  D.div0.init(ctx->n[0]);
  D.div1.init(ctx->n[1]);
  return D;
}

// The vector flush needs 4-aligned tile columns (l_x >= 2) and an x extent
// that is a multiple of 4 (so a wrapped group stays aligned); the field must
// start on a 16-byte (float) or 8-byte (bfloat16) boundary.
inline bool spread_vec(const mls_ctx* ctx) { return ctx->tiles.l[0] >= 2 && ctx->n[0] % 4 == 0; }
inline bool spread_vec_aligned(const mls_ctx* ctx, const void* f) {
  const uintptr_t mask = ctx->opt.field == MLS_F32 ? 15 : 7;
  return spread_vec(ctx) && (reinterpret_cast<uintptr_t>(f) & mask) == 0;
}

}  // namespace mls
