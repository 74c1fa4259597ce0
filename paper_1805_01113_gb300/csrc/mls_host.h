// Host-side state of the MLS transfer library and the kernel launchers the
// C ABI (mls_api.cu) calls.  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mls.h"
#include "mls_device.cuh"

struct mls_kernel_timer {
  const char* name;
  int64_t launches;
  double total_ms;
};

struct mls_event_pair {
  int timer;
  cudaEvent_t start, stop;
};

struct mls_ctx {
  mls_options opt;
  int device;
  int n[3];
  int periodic[3];
  int uniform[3];
  // Grid on the device in both precisions (faces n+1, widths n per axis).
  double* faces_d[3];
  double* widths_d[3];
  float* faces_f[3];
  float* widths_f[3];
  int* bucket_d[3];      // non-uniform axes: cell of each of nbk equal buckets (device), else nullptr
  int nbk[3];
  std::vector<double> faces_host[3];
  mls::Tiles tiles;
  // Fast-MLS table, real[n_classes][n_sub^3][27]; class axis -1 when uniform.
  void* table;
  int64_t n_classes;
  int class_axis;
  // Persistent grid of the spreading kernel (blocks resident on the device).
  int spread_grid;
  int spread_threads;
  int interp_grid;       // persistent grid of the tile-organised interpolation
  int force_grid;        // persistent grid of the fused direct-forcing kernel (0: composed path)
  int collision_grid;    // persistent grid of the collision detection
  int fast_smem_grid;    // persistent grid of the shared-memory fast-MLS build (0: not used)
  int sort_grid;         // persistent grid of the in-tile sort by home cell (0: tiles too large, no sort)
  void* refine_ws;       // refinement workspace (grown on demand)
  int64_t refine_ws_bytes;
  // Learned surrogate: float32 parameters and the packed bfloat16 copy.
  float* mlp_theta;
  unsigned char* mlp_pack;
  // Per-kernel timing.
  int timing;
  std::vector<mls_kernel_timer> timers;
  std::vector<mls_event_pair> events;
  size_t events_used;
};

struct mls_transfer {
  mls_ctx* ctx;
  int64_t cap;
  int64_t M;
  int method;
  void* phi;         // real[27][cap]
  void* c;           // real[cap]
  int32_t* home;     // [cap] tile order
  int32_t* perm;     // [cap] tile order -> caller index
  int32_t* key;      // [cap] caller order: tile bin
  int32_t* rank;     // [cap] caller order: rank inside the bin
  int32_t* counts;   // [nbins]
  int32_t* offsets;  // [nbins]
  int32_t* items;    // [nbins]: non-empty spreading tiles (bin ids, ascending), dropped bin excluded
  int32_t* n_items;  // [1]: number of entries of items
  int32_t* tile_sums;  // [2 * ntiles]: per scan tile, marker sums then non-empty-bin sums
  int ntiles;        // scan tiles over the bins
  unsigned long long* status;  // [4] dropped, nonfinite, refined_fp64, spare
  // Markers already prepared and located for the next build, piece by piece
  // (mls_marker_prep_locate): their arrays, count and the end of the pieces
  // so far.  pre_M < 0: none.
  const void* pre_x;
  const void* pre_area;
  int64_t pre_M;
  int64_t pre_done;
};

namespace mls {

constexpr int kScanTile = 4096;       // bins per scan tile
constexpr int kScanMaxTiles = 8192;   // bins <= 32 Mi
constexpr int kBlock = 256;           // threads per block of the per-marker kernels
constexpr int kBlockF64 = 64;         // the same for the double-precision builds and gradient (FP64-bound:
                                      // small workloads should spread over many SMs)
constexpr int kSpreadThreads = 128;   // threads per block of the spreading kernel
constexpr int kForceThreads = 256;    // threads per block of the fused direct-forcing pass on tiles of at least
                                      // 2^9 cells (smaller tiles: kSpreadThreads)
constexpr int kTableRow = 28;         // fast-MLS table row: 27 shape-function values + 1 pad (16-byte rows)
constexpr int kInterpThreads = 128;   // threads per block of the tile-organised interpolation
constexpr int kSortThreads = 256;     // threads per block of the in-tile sort (a warp per tile)
constexpr int kSortCellsLog2 = 12;    // tiles of up to 2^12 cells are sorted by home cell

// Raises a kernel's dynamic shared-memory limit to at least `bytes` (above the
// 48 KB default).  The limit belongs to the kernel, shared by every context of
// the process, so it is only ever raised: a context with smaller tiles must
// not lower it under one configured earlier.
inline cudaError_t raise_smem_limit(const void* kernel, int bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if (fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// Fast-MLS table shape: sets class_axis and n_classes (MLS_ERR_UNSUPPORTED for
// more than one non-uniform axis); bytes of the table for that shape.
int fast_table_layout(mls_ctx* ctx);
size_t fast_table_bytes(const mls_ctx* ctx);

// Phase helpers: every call opens and closes an NVTX range named after the
// phase; CUDA events are recorded only when ctx->timing is on.
int timer_begin(mls_ctx* ctx, const char* name, cudaStream_t s);
void timer_end(mls_ctx* ctx, int slot, cudaStream_t s);

template <typename R> Grid<R> device_grid(const mls_ctx* ctx);

// Launchers; each returns cudaGetLastError() after enqueueing.
cudaError_t launch_prep(int real, const void* V, int64_t nv, const int32_t* tri, int64_t t0, int64_t t1,
                        int64_t nt, void* x, void* area, cudaStream_t s);
cudaError_t launch_locate(const mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M,
                          cudaStream_t s);
cudaError_t launch_prep_locate(const mls_ctx* ctx, mls_transfer* T, const void* V, int64_t nv, const int32_t* tri,
                               int64_t nt, int64_t t0, int64_t t1, void* x, void* area, cudaStream_t s);
cudaError_t launch_scan(mls_transfer* T, int nbins, cudaStream_t s, mls_ctx* ctx);
cudaError_t launch_scatter(const mls_ctx* ctx, mls_transfer* T, int64_t M, cudaStream_t s);
bool tile_sort_on(const mls_ctx* ctx);
cudaError_t launch_tile_sort(const mls_ctx* ctx, mls_transfer* T, int64_t M, cudaStream_t s);
cudaError_t sort_configure(mls_ctx* ctx);
cudaError_t launch_build_exact(const mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M,
                               cudaStream_t s);
cudaError_t launch_build_fast(const mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M,
                              cudaStream_t s);
// The exact build with the interpolation fused in; with F, also the direct
// forcing F = (Vb - U) / dt (U may then be nullptr).
cudaError_t launch_build_exact_interp(const mls_ctx* ctx, mls_transfer* T, const void* x, const void* area,
                                      int64_t M, const void* u, void* U, cudaStream_t s, const void* Vb = nullptr,
                                      double dt = 0.0, void* F = nullptr);
cudaError_t launch_fast_table(mls_ctx* ctx, cudaStream_t s);
cudaError_t launch_direct_forcing(const mls_ctx* ctx, const mls_transfer* T, const void* u, const void* Vb,
                                  double dt, void* U, void* F, void* f, cudaStream_t s);
cudaError_t force_configure(mls_ctx* ctx);
cudaError_t launch_collisions(const mls_ctx* ctx, const mls_transfer* T, const int32_t* body, int32_t* flag,
                              int32_t* coll, unsigned long long* n_colliding, cudaStream_t s);
cudaError_t collision_configure(mls_ctx* ctx);
cudaError_t build_configure(mls_ctx* ctx);
int64_t refine_workspace_bytes(int64_t nt);
cudaError_t launch_refine(const mls_ctx* ctx, const void* V, int64_t nv, const int32_t* tri, int64_t nt,
                          double ratio, int max_level, int64_t capacity, void* x, void* area, int32_t* parent,
                          int32_t* level, void* ws, int64_t* total_host, cudaStream_t s);
cudaError_t launch_interp_gradient(const mls_ctx* ctx, const mls_transfer* T, const void* x, const void* u, void* G,
                                   cudaStream_t s);
cudaError_t launch_interp(const mls_ctx* ctx, const mls_transfer* T, const void* u, void* U, cudaStream_t s);
cudaError_t launch_spread(const mls_ctx* ctx, const mls_transfer* T, const void* F, void* f, cudaStream_t s);
// Surrogate (k_mlp.cu, mls_surrogate_api.cu).  surrogate_check: MLS_OK when the
// context can hold surrogate parameters, else the error (message set).
int surrogate_check(mls_ctx* ctx, const char* who);
void mlp_init_params(uint64_t seed, float* theta);
int surrogate_class_axis(mls_ctx* ctx);
cudaError_t mlp_configure();
size_t mlp_pack_bytes();
size_t mlp_train_floats(int B);
cudaError_t launch_mlp_samples(const mls_ctx* ctx, int64_t first, int64_t count, uint64_t seed, float* X, float* T,
                               cudaStream_t s);
cudaError_t launch_mlp_grad(const float* theta, const float* X, const float* T, int64_t n_all, int B, bool gather,
                            uint64_t draw_base, uint64_t seed, float* work, float* grad, float* loss_sum,
                            cudaStream_t s);
cudaError_t launch_adam(float* theta, const float* grad, float* m, float* v, float lr, float bc1, float bc2,
                        cudaStream_t s);
cudaError_t launch_scale1(float* v, float s, cudaStream_t st);
cudaError_t launch_mlp_pack(const float* theta, unsigned char* pack, cudaStream_t s);
cudaError_t launch_mlp_forward(const float* theta, const unsigned char* pack, const float* X, int B, int mode,
                               float* Y, cudaStream_t s);
cudaError_t launch_build_surrogate(const mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M,
                                   cudaStream_t s);

size_t spread_smem_bytes(const mls_ctx* ctx);
cudaError_t spread_configure(mls_ctx* ctx);


}  // namespace mls
