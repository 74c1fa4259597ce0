// Euler-to-Lagrange interpolation (gather) and Lagrange-to-Euler spreading
// (scatter through shared-memory tile accumulators).
#include "mls_host.h"

namespace mls {

template <typename FT> __device__ __forceinline__ float to_f(FT v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename R, typename FT> __device__ __forceinline__ R load_field(const FT* p) {
  return (R)to_f<FT>(__ldg(p));
}
template <> __device__ __forceinline__ double load_field<double, double>(const double* p) { return __ldg(p); }

template <typename R, typename FT> __device__ __forceinline__ void add_field(FT* p, R v);
template <> __device__ __forceinline__ void add_field<double, double>(double* p, double v) { atomicAdd(p, v); }
template <> __device__ __forceinline__ void add_field<float, float>(float* p, float v) { atomicAdd(p, v); }
template <> __device__ __forceinline__ void add_field<float, __nv_bfloat16>(__nv_bfloat16* p, float v) {
  atomicAdd(p, __float2bfloat16_rn(v));
}

struct Dims {
  int n[3];
  int periodic[3];
};

__device__ __forceinline__ void decode_home(int32_t h, const Dims& D, int i[3]) {
  i[0] = h % D.n[0];
  const int r = h / D.n[0];
  i[1] = r % D.n[1];
  i[2] = r / D.n[1];
}

// U_l = sum_k phi_k^l u_k for the 3 components (text after Eq. 6).  One
// thread per stored marker; the 27 phi values are read with unit stride
// across the warp, the field through the read-only path.
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

// f_k += sum_l c_l phi_k^l F_l (text after Eq. 7).  A block takes 256
// consecutive stored markers, which are grouped by spreading tile.  For each
// run of markers of one tile it zeroes a shared-memory accumulator covering
// the tile plus a one-cell halo, adds the 81 contributions of every marker
// with shared-memory atomics, then adds each non-zero accumulator cell to f
// with one global atomic per component.
template <typename R, typename FT>
__global__ void __launch_bounds__(kBlock) k_spread(Dims D, Tiles tl, const R* __restrict__ phi,
                                                   const R* __restrict__ cl, const int32_t* __restrict__ home,
                                                   const int32_t* __restrict__ perm, int64_t M, int64_t cap,
                                                   const R* __restrict__ F, FT* __restrict__ f) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* acc = reinterpret_cast<R*>(smem_raw);
  __shared__ int s_key[kBlock];
  const int AX = (1 << tl.l[0]) + 2, AY = (1 << tl.l[1]) + 2, AZ = (1 << tl.l[2]) + 2;
  const int ACC = AX * AY * AZ;
  const int tid = threadIdx.x;
  const int64_t j = (int64_t)blockIdx.x * kBlock + tid;

  int key = INT_MAX;
  int i[3] = {0, 0, 0};
  R v0 = R(0), v1 = R(0), v2 = R(0);
  if (j < M) {
    const int32_t h = home[j];
    if (h >= 0) {
      decode_home(h, D, i);
      key = (((i[2] >> tl.l[2]) * tl.nb[1]) + (i[1] >> tl.l[1])) * tl.nb[0] + (i[0] >> tl.l[0]);
      const int64_t m = perm[j];
      const R c = cl[j];
      v0 = c * F[m];
      v1 = c * F[M + m];
      v2 = c * F[2 * M + m];
    }
  }
  s_key[tid] = key;
  __syncthreads();
  const int64_t N = (int64_t)D.n[0] * D.n[1] * D.n[2];

  int start = 0;
  while (start < kBlock) {
    const int cur = s_key[start];
    if (cur == INT_MAX) break;
    const int bx = cur % tl.nb[0], by = (cur / tl.nb[0]) % tl.nb[1], bz = cur / (tl.nb[0] * tl.nb[1]);
    const int ox = bx << tl.l[0], oy = by << tl.l[1], oz = bz << tl.l[2];
    for (int e = tid; e < 3 * ACC; e += kBlock) acc[e] = R(0);
    __syncthreads();
    if (key == cur) {
      const int lx = i[0] - ox, ly = i[1] - oy, lz = i[2] - oz;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const R p = phi[(9 * c + 3 * b + a) * cap + j];
            const int li = ((lz + c) * AY + (ly + b)) * AX + (lx + a);
            atomicAdd(&acc[li], p * v0);
            atomicAdd(&acc[ACC + li], p * v1);
            atomicAdd(&acc[2 * ACC + li], p * v2);
          }
    }
    __syncthreads();
    for (int e = tid; e < ACC; e += kBlock) {
      const R a0 = acc[e], a1 = acc[ACC + e], a2 = acc[2 * ACC + e];
      if (a0 != R(0) || a1 != R(0) || a2 != R(0)) {
        const int ex = e % AX, ey = (e / AX) % AY, ez = e / (AX * AY);
        const int gx = wrap(ox - 1 + ex, D.n[0], D.periodic[0]);
        const int gy = wrap(oy - 1 + ey, D.n[1], D.periodic[1]);
        const int gz = wrap(oz - 1 + ez, D.n[2], D.periodic[2]);
        const int64_t o = ((int64_t)gz * D.n[1] + gy) * D.n[0] + gx;
        if (a0 != R(0)) add_field<R, FT>(f + o, a0);
        if (a1 != R(0)) add_field<R, FT>(f + N + o, a1);
        if (a2 != R(0)) add_field<R, FT>(f + 2 * N + o, a2);
      }
    }
    start += __syncthreads_count(key == cur);
  }
}

static Dims dims_of(const mls_ctx* ctx) {
  Dims D;
  for (int d = 0; d < 3; ++d) {
    D.n[d] = ctx->n[d];
    D.periodic[d] = ctx->periodic[d];
  }
  return D;
}

size_t spread_smem_bytes(const mls_ctx* ctx) {
  const size_t acc = (size_t)((1 << ctx->tiles.l[0]) + 2) * ((1 << ctx->tiles.l[1]) + 2) *
                     ((1 << ctx->tiles.l[2]) + 2);
  return 3 * acc * (ctx->opt.real == MLS_F64 ? sizeof(double) : sizeof(float));
}

cudaError_t spread_configure(const mls_ctx* ctx) {
  const int smem = (int)spread_smem_bytes(ctx);
  if (smem <= 48 * 1024) return cudaSuccess;
  if (ctx->opt.real == MLS_F64)
    return cudaFuncSetAttribute(k_spread<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (ctx->opt.field == MLS_F32)
    return cudaFuncSetAttribute(k_spread<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return cudaFuncSetAttribute(k_spread<float, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_interp(const mls_ctx* ctx, const mls_transfer* T, const void* u, void* U, cudaStream_t s) {
  if (T->M == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((T->M + kBlock - 1) / kBlock);
  const Dims D = dims_of(ctx);
  if (ctx->opt.real == MLS_F64)
    k_interp<double, double><<<grid, kBlock, 0, s>>>(D, (const double*)T->phi, T->home, T->perm, T->M, T->cap,
                                                     (const double*)u, (double*)U);
  else if (ctx->opt.field == MLS_F32)
    k_interp<float, float><<<grid, kBlock, 0, s>>>(D, (const float*)T->phi, T->home, T->perm, T->M, T->cap,
                                                   (const float*)u, (float*)U);
  else
    k_interp<float, __nv_bfloat16><<<grid, kBlock, 0, s>>>(D, (const float*)T->phi, T->home, T->perm, T->M,
                                                           T->cap, (const __nv_bfloat16*)u, (float*)U);
  return cudaGetLastError();
}

cudaError_t launch_spread(const mls_ctx* ctx, const mls_transfer* T, const void* F, void* f, cudaStream_t s) {
  if (T->M == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((T->M + kBlock - 1) / kBlock);
  const Dims D = dims_of(ctx);
  const size_t smem = spread_smem_bytes(ctx);
  if (ctx->opt.real == MLS_F64)
    k_spread<double, double><<<grid, kBlock, smem, s>>>(D, ctx->tiles, (const double*)T->phi, (const double*)T->c,
                                                        T->home, T->perm, T->M, T->cap, (const double*)F,
                                                        (double*)f);
  else if (ctx->opt.field == MLS_F32)
    k_spread<float, float><<<grid, kBlock, smem, s>>>(D, ctx->tiles, (const float*)T->phi, (const float*)T->c,
                                                      T->home, T->perm, T->M, T->cap, (const float*)F, (float*)f);
  else
    k_spread<float, __nv_bfloat16><<<grid, kBlock, smem, s>>>(D, ctx->tiles, (const float*)T->phi,
                                                              (const float*)T->c, T->home, T->perm, T->M, T->cap,
                                                              (const float*)F, (__nv_bfloat16*)f);
  return cudaGetLastError();
}

}  // namespace mls
