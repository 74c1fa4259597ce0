// Fused direct-forcing transfer: interpolation, the IBM force and spreading
// in one pass over the spreading tiles, reading phi once.
#include "force_tile.cuh"

namespace mls {

// F_l = (V_b,l - U_l) / dt in place over U, for the composed (unfused) path:
// tile order j, caller index perm[j]; markers without support (home < 0)
// get F = 0.
template <typename R>
__global__ void __launch_bounds__(kBlock) k_force_from_u(const int32_t* __restrict__ home,
                                                         const int32_t* __restrict__ perm, int64_t M,
                                                         const R* __restrict__ Vb, R inv_dt, R* __restrict__ UF) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const int64_t m = perm[j];
  const bool ok = home[j] >= 0;
#pragma unroll
  for (int q = 0; q < 3; ++q) UF[q * M + m] = ok ? (Vb[q * M + m] - UF[q * M + m]) * inv_dt : R(0);
}

const void* force_kernel_128(bool bf, bool vec, int lx, int ly, int lz) {
  constexpr int NT = kSpreadThreads;
  return bf ? (vec ? force_kernel<__nv_bfloat16, true, NT>(lx, ly, lz) : force_kernel<__nv_bfloat16, false, NT>(lx, ly, lz))
            : (vec ? force_kernel<float, true, NT>(lx, ly, lz) : force_kernel<float, false, NT>(lx, ly, lz));
}

// Threads per block (= markers per chunk) of the fused pass: 256 for tiles of
// at least 2^9 cells, which hold enough markers to fill such chunks (3.88
// against 4.21 ms on the 10^4-body workload, tiles 3,3,3), else 128 (tiles
// 3,3,2 on c2 leave half of 256-marker chunks empty).
static int force_threads(const mls_ctx* ctx) {
  return ctx->tiles.l[0] + ctx->tiles.l[1] + ctx->tiles.l[2] >= 9 ? kForceThreads : kSpreadThreads;
}

template <typename FT, bool VEC>
static const void* force_kernel_for(const mls_ctx* ctx) {
  const int* l = ctx->tiles.l;
  constexpr bool bf = sizeof(FT) == 2;
  return force_threads(ctx) == kForceThreads ? force_kernel_256(bf, VEC, l[0], l[1], l[2])
                                             : force_kernel_128(bf, VEC, l[0], l[1], l[2]);
}

size_t force_smem_bytes(const mls_ctx* ctx) {
  const int* l = ctx->tiles.l;
  return (size_t)ForceSmem(l[0], l[1], l[2], spread_vec(ctx)).total;
}

static cudaError_t force_configure_one(mls_ctx* ctx, const void* k, int smem) {
  cudaError_t e;
  if ((e = raise_smem_limit(k, smem)) != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, force_threads(ctx), smem)) != cudaSuccess)
    return e;
  ctx->force_grid = (per_sm > 0 ? per_sm : 1) * sms;
  return cudaSuccess;
}

// Grid of the fused kernel; a context whose fused brick and accumulator do
// not fit one block's shared memory gets force_grid = 0 and composes the
// separate kernels instead.
cudaError_t force_configure(mls_ctx* ctx) {
  ctx->force_grid = 0;
  if (ctx->opt.real == MLS_F64) return cudaSuccess;
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  if (e != cudaSuccess) return e;
  const int smem = (int)force_smem_bytes(ctx);
  if (smem > optin) return cudaSuccess;
  const bool bf = ctx->opt.field == MLS_BF16;
  if (spread_vec(ctx)) {
    e = force_configure_one(ctx, bf ? force_kernel_for<__nv_bfloat16, false>(ctx) : force_kernel_for<float, false>(ctx),
                            smem);
    if (e != cudaSuccess) return e;
    return force_configure_one(ctx, bf ? force_kernel_for<__nv_bfloat16, true>(ctx) : force_kernel_for<float, true>(ctx),
                               smem);
  }
  return force_configure_one(ctx, bf ? force_kernel_for<__nv_bfloat16, false>(ctx) : force_kernel_for<float, false>(ctx),
                             smem);
}

cudaError_t launch_direct_forcing(const mls_ctx* ctx, const mls_transfer* T, const void* u, const void* Vb,
                                  double dt, void* U, void* F, void* f, cudaStream_t s) {
  if (T->M == 0) return cudaSuccess;
  if (ctx->opt.real == MLS_F64 || ctx->force_grid == 0) {
    // Composition of the separate kernels: interpolation into U (or F),
    // the force in place, spreading of F.
    void* UF = U ? U : F;
    cudaError_t e = launch_interp(ctx, T, u, UF, s);
    if (e != cudaSuccess) return e;
    if (U && (e = cudaMemcpyAsync(F, U, (size_t)3 * T->M * (ctx->opt.real == MLS_F64 ? 8 : 4),
                                  cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
    const unsigned grid = (unsigned)((T->M + kBlock - 1) / kBlock);
    if (ctx->opt.real == MLS_F64)
      k_force_from_u<double><<<grid, kBlock, 0, s>>>(T->home, T->perm, T->M, (const double*)Vb, 1.0 / dt,
                                                     (double*)F);
    else
      k_force_from_u<float><<<grid, kBlock, 0, s>>>(T->home, T->perm, T->M, (const float*)Vb, (float)(1.0 / dt),
                                                    (float*)F);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_spread(ctx, T, F, f, s);
  }
  Dims D = dims_of(ctx);
  Tiles tl = ctx->tiles;
  const float* phi = (const float*)T->phi;
  const float* c = (const float*)T->c;
  int64_t M = T->M, cap = T->cap;
  float inv_dt = (float)(1.0 / dt);
  const bool vec = spread_vec_aligned(ctx, f);
  const bool bf = ctx->opt.field == MLS_BF16;
  const void* k = bf ? (vec ? force_kernel_for<__nv_bfloat16, true>(ctx) : force_kernel_for<__nv_bfloat16, false>(ctx))
                     : (vec ? force_kernel_for<float, true>(ctx) : force_kernel_for<float, false>(ctx));
  void* args[] = {&D, &tl, (void*)&phi, (void*)&c, (void*)&T->home, (void*)&T->perm, (void*)&T->items,
                  (void*)&T->n_items, (void*)&T->offsets, (void*)&T->counts, &M, &cap, (void*)&u, (void*)&Vb,
                  &inv_dt, &U, &F, &f};
  return cudaLaunchKernel(k, dim3(ctx->force_grid), dim3(force_threads(ctx)), args, force_smem_bytes(ctx), s);
}

}  // namespace mls
