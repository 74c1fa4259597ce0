// mls_build_transfer_noalloc: the build of mls_build_transfer for callers that
// cannot allocate device memory when they build.  The outputs go to buffers
// the caller owns; the tile-sort workspace (bin keys and ranks, bin counts,
// bin offsets, the tile list, scan tile sums, counters) lives in one file-scope device array
// of fixed size instead of a transfer handle.  The kernels are the same ones
// mls_build_transfer launches.
#include <mutex>

#include "mls_host.h"

namespace {

using mls::kScanTile;

constexpr int64_t kMaxMarkers = MLS_NOALLOC_MAX_MARKERS;
constexpr int64_t kMaxBins = MLS_NOALLOC_MAX_BINS;
constexpr int64_t kMaxTiles = (kMaxBins + kScanTile - 1) / kScanTile;

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kOffKey = 0;
constexpr size_t kOffRank = kOffKey + align256(kMaxMarkers * 4);
constexpr size_t kOffCounts = kOffRank + align256(kMaxMarkers * 4);
constexpr size_t kOffOffsets = kOffCounts + align256(kMaxBins * 4);
constexpr size_t kOffItems = kOffOffsets + align256(kMaxBins * 4);
constexpr size_t kOffTiles = kOffItems + align256(kMaxBins * 4);
constexpr size_t kOffStatus = kOffTiles + align256(2 * kMaxTiles * 4);
constexpr size_t kOffNItems = kOffStatus + 256;
constexpr size_t kScratchBytes = kOffNItems + 256;
static_assert(kScratchBytes == MLS_NOALLOC_SCRATCH_BYTES, "header and layout disagree");

// The workspace.  Every device that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host code cannot use g_scratch's name as a device address; its address on
// each device is looked up once, with that device current, and cached here
// for the life of the process (the device's primary context is assumed to
// live as long; after cudaDeviceReset the cached address would be stale).
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

int scratch_on_current_device(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    mls::set_error("mls_build_transfer_noalloc: device index out of range");
    return MLS_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return mls::cuda_fail(e, "mls_build_transfer_noalloc: cudaGetSymbolAddress");
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return MLS_OK;
}

int fail(int code, const char* msg) {
  mls::set_error(msg);
  return code;
}

}  // namespace

extern "C" int mls_build_transfer_noalloc(mls_ctx* ctx, const void* x, const void* area, int64_t M,
                                          int32_t method, void* phi, void* c, int32_t* home, int32_t* perm,
                                          int64_t ld_phi, void* stream) {
  if (!ctx) return fail(MLS_ERR_INVALID_ARG, "mls_build_transfer_noalloc: NULL context");
  if (M < 0) return fail(MLS_ERR_INVALID_ARG, "mls_build_transfer_noalloc: negative M");
  if (M > kMaxMarkers)
    return fail(MLS_ERR_CAPACITY, "mls_build_transfer_noalloc: M exceeds MLS_NOALLOC_MAX_MARKERS (262144)");
  if (ctx->tiles.nbins > kMaxBins)
    return fail(MLS_ERR_CAPACITY,
                "mls_build_transfer_noalloc: the grid has more spreading tiles than MLS_NOALLOC_MAX_BINS - 1; "
                "use a larger brick_log2");
  if (method == MLS_SURROGATE)
    return fail(MLS_ERR_UNSUPPORTED,
                "mls_build_transfer_noalloc: the surrogate is not offered without allocation; use MLS_EXACT or "
                "MLS_FAST, or mls_build_transfer");
  if (method != MLS_EXACT && method != MLS_FAST)
    return fail(MLS_ERR_INVALID_ARG, "mls_build_transfer_noalloc: unknown method");
  if (M > 0 && (!x || !area || !phi || !c || !home || !perm))
    return fail(MLS_ERR_INVALID_ARG, "mls_build_transfer_noalloc: NULL array");
  if (ld_phi < M || ld_phi > 0x7fffffffLL - 1)
    return fail(MLS_ERR_INVALID_ARG, "mls_build_transfer_noalloc: ld_phi must be in [M, 2^31-2]");
  if (method == MLS_FAST && !ctx->table)
    return fail(MLS_ERR_UNSUPPORTED,
                "mls_build_transfer_noalloc: the fast-MLS table does not exist yet; call mls_fast_table first");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return mls::cuda_fail(e, "mls_build_transfer_noalloc: cudaGetDevice");
  if (dev != ctx->device)
    return fail(MLS_ERR_INVALID_ARG, "mls_build_transfer_noalloc: the context's device is not current");
  unsigned char* s = nullptr;
  int rc = scratch_on_current_device(dev, &s);
  if (rc != MLS_OK) return rc;

  mls_transfer T;
  T.ctx = ctx;
  T.cap = ld_phi;
  T.M = M;
  T.method = method;
  T.phi = phi;
  T.c = c;
  T.home = home;
  T.perm = perm;
  T.key = reinterpret_cast<int32_t*>(s + kOffKey);
  T.rank = reinterpret_cast<int32_t*>(s + kOffRank);
  T.counts = reinterpret_cast<int32_t*>(s + kOffCounts);
  T.offsets = reinterpret_cast<int32_t*>(s + kOffOffsets);
  T.items = reinterpret_cast<int32_t*>(s + kOffItems);
  T.n_items = reinterpret_cast<int32_t*>(s + kOffNItems);
  T.tile_sums = reinterpret_cast<int32_t*>(s + kOffTiles);
  T.ntiles = (ctx->tiles.nbins + kScanTile - 1) / kScanTile;
  T.status = reinterpret_cast<unsigned long long*>(s + kOffStatus);

  cudaStream_t st = (cudaStream_t)stream;
  // The array keeps the previous call's contents: clear what must start at zero.
  if ((e = cudaMemsetAsync(T.status, 0, 4 * sizeof(unsigned long long), st)) != cudaSuccess)
    return mls::cuda_fail(e, "mls_build_transfer_noalloc: counter reset");
  if (M == 0) return MLS_OK;
  if ((e = cudaMemsetAsync(T.counts, 0, (size_t)ctx->tiles.nbins * 4, st)) != cudaSuccess)
    return mls::cuda_fail(e, "mls_build_transfer_noalloc: bin reset");
  if ((e = mls::launch_locate(ctx, &T, x, area, M, st)) != cudaSuccess)
    return mls::cuda_fail(e, "mls_build_transfer_noalloc: locate");
  if ((e = mls::launch_scan(&T, ctx->tiles.nbins, st, nullptr)) != cudaSuccess)
    return mls::cuda_fail(e, "mls_build_transfer_noalloc: scan");
  if ((e = mls::launch_scatter(ctx, &T, M, st)) != cudaSuccess)
    return mls::cuda_fail(e, "mls_build_transfer_noalloc: scatter");
  if ((e = mls::launch_tile_sort(ctx, &T, M, st)) != cudaSuccess)
    return mls::cuda_fail(e, "mls_build_transfer_noalloc: tile sort");
  e = method == MLS_EXACT ? mls::launch_build_exact(ctx, &T, x, area, M, st)
                          : mls::launch_build_fast(ctx, &T, x, area, M, st);
  if (e != cudaSuccess) return mls::cuda_fail(e, "mls_build_transfer_noalloc: build");
  return MLS_OK;
}
