// C ABI of the MLS transfer library (see include/mls.h): argument checks,
// device memory ownership, and the kernel sequence of each call.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "mls_host.h"

namespace mls {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return MLS_ERR_CUDA;
}

static int invalid(const char* msg) {
  set_error(msg);
  return MLS_ERR_INVALID_ARG;
}

template <typename R>
Grid<R> device_grid(const mls_ctx* ctx) {
  Grid<R> g;
  for (int d = 0; d < 3; ++d) {
    Axis<R>& a = g.ax[d];
    const std::vector<double>& f = ctx->faces_host[d];
    if (sizeof(R) == sizeof(double)) {
      a.faces = (const R*)ctx->faces_d[d];
      a.widths = (const R*)ctx->widths_d[d];
    } else {
      a.faces = (const R*)ctx->faces_f[d];
      a.widths = (const R*)ctx->widths_f[d];
    }
    a.n = ctx->n[d];
    a.periodic = ctx->periodic[d];
    a.uniform = ctx->uniform[d];
    a.lo = (R)f.front();
    a.hi = (R)f.back();
    a.h = (R)(f[1] - f[0]);
    a.inv_h = (R)(1.0 / (f[1] - f[0]));
    a.bucket = ctx->bucket_d[d];
    a.nbk = ctx->nbk[d];
    a.inv_bw = ctx->nbk[d] > 0 ? (R)((double)ctx->nbk[d] / (f.back() - f.front())) : R(0);
  }
  return g;
}
template Grid<float> device_grid<float>(const mls_ctx*);
template Grid<double> device_grid<double>(const mls_ctx*);

int timer_begin(mls_ctx* ctx, const char* name, cudaStream_t s) {
  // Host-side range named after the phase, for Nsight tools (`ncu --nvtx`);
  // without a tool attached the call only tests a function pointer.
  nvtxRangePushA(name);
  if (!ctx || !ctx->timing) return -1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return -1;
  int t = -1;
  for (size_t q = 0; q < ctx->timers.size(); ++q)
    if (ctx->timers[q].name == name || std::strcmp(ctx->timers[q].name, name) == 0) t = (int)q;
  if (t < 0) {
    ctx->timers.push_back({name, 0, 0.0});
    t = (int)ctx->timers.size() - 1;
  }
  if (ctx->events_used == ctx->events.size()) {
    mls_event_pair p;
    p.timer = t;
    if (cudaEventCreate(&p.start) != cudaSuccess) return -1;
    if (cudaEventCreate(&p.stop) != cudaSuccess) {
      cudaEventDestroy(p.start);
      return -1;
    }
    ctx->events.push_back(p);
  }
  const int slot = (int)ctx->events_used++;
  ctx->events[slot].timer = t;
  cudaEventRecord(ctx->events[slot].start, s);
  return slot;
}

void timer_end(mls_ctx* ctx, int slot, cudaStream_t s) {
  nvtxRangePop();
  if (slot < 0) return;
  cudaEventRecord(ctx->events[slot].stop, s);
}

int fast_table_layout(mls_ctx* ctx) {
  int axis = -1, nonuni = 0;
  for (int d = 0; d < 3; ++d)
    if (!ctx->uniform[d]) {
      axis = d;
      ++nonuni;
    }
  if (nonuni > 1) {
    set_error("fast-MLS tables need at most one non-uniform axis");
    return MLS_ERR_UNSUPPORTED;
  }
  ctx->class_axis = axis;
  ctx->n_classes = axis < 0 ? 1 : ctx->n[axis];
  return MLS_OK;
}

size_t fast_table_bytes(const mls_ctx* ctx) {
  const int64_t S3 = (int64_t)ctx->opt.n_sub * ctx->opt.n_sub * ctx->opt.n_sub;
  const size_t rs = ctx->opt.real == MLS_F64 ? sizeof(double) : sizeof(float);
  return (size_t)ctx->n_classes * S3 * kTableRow * rs;
}

}  // namespace mls

using namespace mls;

extern "C" {

const char* mls_last_error(void) { return g_last_error.c_str(); }

const char* mls_strerror(int32_t code) {
  switch (code) {
    case MLS_OK: return "ok";
    case MLS_ERR_INVALID_ARG: return "invalid argument";
    case MLS_ERR_CAPACITY: return "more markers than the transfer handle holds";
    case MLS_ERR_UNSUPPORTED: return "unsupported request";
    case MLS_ERR_CUDA: return "CUDA runtime error";
    case MLS_ERR_OUT_OF_DOMAIN: return "markers dropped (outside the grid, non-finite, or support off a wall)";
    default: return "unknown status";
  }
}

int mls_options_default(mls_options* opt) {
  if (!opt) return invalid("mls_options_default: NULL");
  opt->real = MLS_F32;
  opt->field = MLS_F32;
  opt->eps = 1.0;
  opt->n_sub = 9;
  opt->brick_log2[0] = opt->brick_log2[1] = opt->brick_log2[2] = 3;
  opt->cond_max = 1e6;
  opt->refine = 1;
  opt->residual_max = 1e-4;
  opt->basis = 4;
  return MLS_OK;
}

static void free_ctx(mls_ctx* c) {
  if (!c) return;
  for (int d = 0; d < 3; ++d) {
    cudaFree(c->faces_d[d]);
    cudaFree(c->widths_d[d]);
    cudaFree(c->faces_f[d]);
    cudaFree(c->widths_f[d]);
  }
  cudaFree(c->table);
  cudaFree(c->mlp_theta);
  cudaFree(c->mlp_pack);
  cudaFree(c->refine_ws);
  for (int d = 0; d < 3; ++d) cudaFree(c->bucket_d[d]);
  for (auto& p : c->events) {
    cudaEventDestroy(p.start);
    cudaEventDestroy(p.stop);
  }
  delete c;
}

int mls_create(const mls_grid* grid, const mls_options* opt_in, mls_ctx** out) {
  if (!grid || !out) return invalid("mls_create: NULL grid or out");
  *out = nullptr;
  mls_options opt;
  if (opt_in) opt = *opt_in; else mls_options_default(&opt);
  if (opt.real != MLS_F64 && opt.real != MLS_F32) return invalid("mls_create: real must be MLS_F64 or MLS_F32");
  if (opt.field != MLS_F64 && opt.field != MLS_F32 && opt.field != MLS_BF16)
    return invalid("mls_create: unknown field type");
  if ((opt.real == MLS_F64) != (opt.field == MLS_F64))
    return invalid("mls_create: double fields need real = MLS_F64 and vice versa");
  if (!(opt.eps > 0.0) || !std::isfinite(opt.eps)) return invalid("mls_create: eps must be positive");
  if (opt.n_sub < 3 || opt.n_sub > 33) return invalid("mls_create: n_sub must be in [3, 33]");
  if (opt.refine < 0 || opt.refine > 2) return invalid("mls_create: refine must be 0, 1 or 2");
  if (!(opt.residual_max > 0.0)) return invalid("mls_create: residual_max must be positive");
  if (opt.basis != 4 && opt.basis != kQuad) return invalid("mls_create: basis must be 4 or 10");
  for (int d = 0; d < 3; ++d)
    if (opt.brick_log2[d] < 1 || opt.brick_log2[d] > 5) return invalid("mls_create: brick_log2 must be in [1, 5]");
  int64_t cells = 1;
  for (int d = 0; d < 3; ++d) {
    if (grid->n[d] < 3) return invalid("mls_create: every axis needs at least 3 cells");
    if (!grid->faces[d]) return invalid("mls_create: NULL faces");
    cells *= grid->n[d];
    for (int i = 0; i < grid->n[d]; ++i)
      if (!(grid->faces[d][i + 1] > grid->faces[d][i]) || !std::isfinite(grid->faces[d][i + 1]))
        return invalid("mls_create: faces must be finite and strictly increasing");
  }
  if (cells >= (int64_t(1) << 31)) return invalid("mls_create: n[0]*n[1]*n[2] must be < 2^31");

  mls_ctx* c = new (std::nothrow) mls_ctx();
  if (!c) return invalid("mls_create: out of host memory");
  c->opt = opt;
  c->table = nullptr;
  c->refine_ws = nullptr;
  c->refine_ws_bytes = 0;
  c->n_classes = 0;
  c->class_axis = -1;
  c->timing = 0;
  c->events_used = 0;
  cudaGetDevice(&c->device);
  int64_t nbins = 1;
  for (int d = 0; d < 3; ++d) {
    const int n = grid->n[d];
    c->n[d] = n;
    c->periodic[d] = grid->periodic[d] ? 1 : 0;
    c->faces_host[d].assign(grid->faces[d], grid->faces[d] + n + 1);
    std::vector<double> w(n);
    std::vector<float> ff(n + 1), wf(n);
    bool uni = true;
    const double w0 = grid->faces[d][1] - grid->faces[d][0];
    for (int i = 0; i < n; ++i) {
      w[i] = grid->faces[d][i + 1] - grid->faces[d][i];
      if (std::fabs(w[i] - w0) > 1e-12 * w0) uni = false;
    }
    for (int i = 0; i <= n; ++i) ff[i] = (float)grid->faces[d][i];
    for (int i = 0; i < n; ++i) wf[i] = ff[i + 1] - ff[i];
    c->uniform[d] = uni ? 1 : 0;
    // Bucket table of a non-uniform axis: 4n equal buckets of [faces[0], faces[n]),
    // each with the cell that contains its lower edge.
    std::vector<int> bk;
    if (!uni) {
      const int nbk = 4 * n;
      bk.resize(nbk);
      const double lo = grid->faces[d][0], span = grid->faces[d][n] - lo;
      int i = 0;
      for (int b = 0; b < nbk; ++b) {
        const double edge = lo + span * (double)b / (double)nbk;
        while (i < n - 1 && grid->faces[d][i + 1] <= edge) ++i;
        bk[b] = i;
      }
      c->nbk[d] = nbk;
    }
    cudaError_t e;
    if ((e = cudaMalloc(&c->faces_d[d], (n + 1) * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&c->widths_d[d], n * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&c->faces_f[d], (n + 1) * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&c->widths_f[d], n * sizeof(float))) != cudaSuccess ||
        (e = cudaMemcpy(c->faces_d[d], grid->faces[d], (n + 1) * sizeof(double), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(c->widths_d[d], w.data(), n * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c->faces_f[d], ff.data(), (n + 1) * sizeof(float), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(c->widths_f[d], wf.data(), n * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (!bk.empty() && ((e = cudaMalloc(&c->bucket_d[d], bk.size() * sizeof(int))) != cudaSuccess ||
                         (e = cudaMemcpy(c->bucket_d[d], bk.data(), bk.size() * sizeof(int),
                                         cudaMemcpyHostToDevice)) != cudaSuccess))) {
      free_ctx(c);
      return cuda_fail(e, "mls_create");
    }
    c->tiles.l[d] = opt.brick_log2[d];
    c->tiles.nb[d] = (n + (1 << opt.brick_log2[d]) - 1) >> opt.brick_log2[d];
    nbins *= c->tiles.nb[d];
  }
  nbins += 1;
  if (nbins > (int64_t)kScanTile * kScanMaxTiles) {
    free_ctx(c);
    return invalid("mls_create: too many spreading tiles; raise brick_log2");
  }
  c->tiles.nbins = (int)nbins;
  if (spread_smem_bytes(c) > 200 * 1024 + 256) {
    free_ctx(c);
    return invalid("mls_create: spreading tile too large for shared memory; lower brick_log2");
  }
  cudaError_t e = spread_configure(c);
  if (e == cudaSuccess) e = force_configure(c);
  if (e == cudaSuccess) e = collision_configure(c);
  if (e == cudaSuccess) e = build_configure(c);
  if (e == cudaSuccess) e = sort_configure(c);
  if (e == cudaSuccess) e = mlp_configure();
  if (e != cudaSuccess) {
    free_ctx(c);
    return cuda_fail(e, "mls_create: kernel configuration");
  }
  *out = c;
  return MLS_OK;
}

int mls_destroy(mls_ctx* ctx) {
  if (!ctx) return invalid("mls_destroy: NULL");
  free_ctx(ctx);
  return MLS_OK;
}

static void free_transfer(mls_transfer* T) {
  if (!T) return;
  cudaFree(T->phi);
  cudaFree(T->c);
  cudaFree(T->home);
  cudaFree(T->perm);
  cudaFree(T->key);
  cudaFree(T->rank);
  cudaFree(T->counts);
  cudaFree(T->offsets);
  cudaFree(T->items);
  cudaFree(T->n_items);
  cudaFree(T->tile_sums);
  cudaFree(T->status);
  delete T;
}

int mls_transfer_create(mls_ctx* ctx, int64_t capacity, mls_transfer** out) {
  if (!ctx || !out) return invalid("mls_transfer_create: NULL argument");
  *out = nullptr;
  if (capacity < 1 || capacity > 0x7fffffffLL - 1) return invalid("mls_transfer_create: capacity must be in [1, 2^31-2]");
  mls_transfer* T = new (std::nothrow) mls_transfer();
  if (!T) return invalid("mls_transfer_create: out of host memory");
  T->ctx = ctx;
  T->cap = capacity;
  T->M = 0;
  T->method = MLS_EXACT;
  T->pre_M = -1;
  const size_t rs = ctx->opt.real == MLS_F64 ? sizeof(double) : sizeof(float);
  const int nbins = ctx->tiles.nbins;
  T->ntiles = (nbins + kScanTile - 1) / kScanTile;
  cudaError_t e;
  if ((e = cudaMalloc(&T->phi, 27 * (size_t)capacity * rs)) != cudaSuccess ||
      (e = cudaMalloc(&T->c, (size_t)capacity * rs)) != cudaSuccess ||
      (e = cudaMalloc(&T->home, (size_t)capacity * 4)) != cudaSuccess ||
      (e = cudaMalloc(&T->perm, (size_t)capacity * 4)) != cudaSuccess ||
      (e = cudaMalloc(&T->key, (size_t)capacity * 4)) != cudaSuccess ||
      (e = cudaMalloc(&T->rank, (size_t)capacity * 4)) != cudaSuccess ||
      (e = cudaMalloc(&T->counts, (size_t)nbins * 4)) != cudaSuccess ||
      (e = cudaMalloc(&T->offsets, (size_t)nbins * 4)) != cudaSuccess ||
      (e = cudaMalloc(&T->items, (size_t)nbins * 4)) != cudaSuccess ||
      (e = cudaMalloc(&T->n_items, 4)) != cudaSuccess ||
      (e = cudaMemset(T->n_items, 0, 4)) != cudaSuccess ||
      (e = cudaMalloc(&T->tile_sums, (size_t)T->ntiles * 2 * 4)) != cudaSuccess ||
      (e = cudaMalloc(&T->status, 4 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMemset(T->status, 0, 4 * sizeof(unsigned long long))) != cudaSuccess) {
    free_transfer(T);
    return cuda_fail(e, "mls_transfer_create");
  }
  *out = T;
  return MLS_OK;
}

int mls_transfer_destroy(mls_transfer* T) {
  if (!T) return invalid("mls_transfer_destroy: NULL");
  free_transfer(T);
  return MLS_OK;
}

int mls_marker_prep_range(mls_ctx* ctx, const void* vertices, int64_t n_vertices, const int32_t* tri,
                          int64_t n_tri, int64_t t_begin, int64_t t_end, void* x, void* area, void* stream) {
  if (!ctx) return invalid("mls_marker_prep: NULL ctx");
  if (n_tri < 0 || n_vertices < 0) return invalid("mls_marker_prep: negative size");
  if (t_begin < 0 || t_begin > t_end || t_end > n_tri)
    return invalid("mls_marker_prep_range: range not within [0, n_tri]");
  if (t_end > t_begin && (!vertices || !tri || !x || !area)) return invalid("mls_marker_prep: NULL pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const int slot = timer_begin(ctx, "marker_prep", s);
  cudaError_t e = launch_prep(ctx->opt.real, vertices, n_vertices, tri, t_begin, t_end, n_tri, x, area, s);
  timer_end(ctx, slot, s);
  if (e != cudaSuccess) return cuda_fail(e, "mls_marker_prep");
  return MLS_OK;
}

int mls_marker_prep(mls_ctx* ctx, const void* vertices, int64_t n_vertices, const int32_t* tri, int64_t n_tri,
                    void* x, void* area, void* stream) {
  return mls_marker_prep_range(ctx, vertices, n_vertices, tri, n_tri, 0, n_tri, x, area, stream);
}

int mls_marker_prep_locate(mls_ctx* ctx, mls_transfer* T, const void* vertices, int64_t n_vertices,
                           const int32_t* tri, int64_t n_tri, int64_t t_begin, int64_t t_end, void* x, void* area,
                           void* stream) {
  if (!ctx || !T) return invalid("mls_marker_prep_locate: NULL handle");
  if (T->ctx != ctx) return invalid("mls_marker_prep_locate: transfer belongs to another context");
  if (n_tri < 0 || n_vertices < 0) return invalid("mls_marker_prep_locate: negative size");
  if (n_tri > T->cap) {
    set_error("mls_marker_prep_locate: n_tri exceeds the transfer capacity");
    return MLS_ERR_CAPACITY;
  }
  if (t_begin < 0 || t_begin > t_end || t_end > n_tri)
    return invalid("mls_marker_prep_locate: range not within [0, n_tri]");
  if (n_tri > 0 && (!vertices || !tri || !x || !area)) return invalid("mls_marker_prep_locate: NULL pointer");
  if (t_begin != 0 &&
      !(T->pre_M == n_tri && T->pre_done == t_begin && T->pre_x == x && T->pre_area == area))
    return invalid("mls_marker_prep_locate: a piece must start at triangle 0 or where the previous piece on this "
                   "transfer ended, with the same n_tri, x and area");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (t_begin == 0) {
    // A new set of markers: the counters and tile bins of the next build start from zero.
    T->pre_M = -1;
    if ((e = cudaMemsetAsync(T->status, 0, 4 * sizeof(unsigned long long), s)) != cudaSuccess)
      return cuda_fail(e, "mls_marker_prep_locate: status reset");
    const int slot = timer_begin(ctx, "bin_reset", s);
    e = cudaMemsetAsync(T->counts, 0, (size_t)ctx->tiles.nbins * 4, s);
    timer_end(ctx, slot, s);
    if (e != cudaSuccess) return cuda_fail(e, "mls_marker_prep_locate: bin reset");
    T->pre_x = x;
    T->pre_area = area;
    T->pre_M = n_tri;
    T->pre_done = 0;
  }
  const int slot = timer_begin(ctx, "prep_locate", s);
  e = launch_prep_locate(ctx, T, vertices, n_vertices, tri, n_tri, t_begin, t_end, x, area, s);
  timer_end(ctx, slot, s);
  if (e != cudaSuccess) {
    T->pre_M = -1;
    return cuda_fail(e, "mls_marker_prep_locate");
  }
  T->pre_done = t_end;
  return MLS_OK;
}

int mls_refine_markers(mls_ctx* ctx, const void* vertices, int64_t n_vertices, const int32_t* tri, int64_t n_tri,
                       double ratio, int32_t max_level, int64_t capacity, void* x, void* area, int32_t* parent,
                       int32_t* level, int64_t* n_markers, void* stream) {
  if (!ctx || !n_markers) return invalid("mls_refine_markers: NULL ctx or n_markers");
  if (n_tri < 0 || n_vertices < 0 || capacity < 0) return invalid("mls_refine_markers: negative size");
  if (!(ratio > 0.0) || !std::isfinite(ratio)) return invalid("mls_refine_markers: ratio must be positive");
  if (max_level < 0 || max_level > 3) return invalid("mls_refine_markers: max_level must be in 0..3");
  if (n_tri > 0 && (!vertices || !tri || !x || !area || !parent))
    return invalid("mls_refine_markers: NULL pointer");
  if (n_tri > ((int64_t)1 << 29)) return invalid("mls_refine_markers: too many triangles");
  *n_markers = 0;
  if (n_tri == 0) return MLS_OK;
  const int64_t need = refine_workspace_bytes(n_tri);
  if (need > ctx->refine_ws_bytes) {
    cudaFree(ctx->refine_ws);
    ctx->refine_ws = nullptr;
    ctx->refine_ws_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->refine_ws, (size_t)need);
    if (e != cudaSuccess) return cuda_fail(e, "mls_refine_markers: workspace");
    ctx->refine_ws_bytes = need;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int slot = timer_begin(ctx, "refine", s);
  int64_t total = 0;
  cudaError_t e = launch_refine(ctx, vertices, n_vertices, tri, n_tri, ratio, max_level, capacity, x, area, parent,
                                level, ctx->refine_ws, &total, s);
  timer_end(ctx, slot, s);
  if (e != cudaSuccess) return cuda_fail(e, "mls_refine_markers");
  *n_markers = total;
  if (total > capacity) {
    set_error("mls_refine_markers: more refined markers than capacity");
    return MLS_ERR_CAPACITY;
  }
  return MLS_OK;
}

static int ensure_table(mls_ctx* ctx, cudaStream_t s) {
  if (ctx->table) return MLS_OK;
  int rc = fast_table_layout(ctx);
  if (rc != MLS_OK) return rc;
  cudaError_t e = cudaMalloc(&ctx->table, fast_table_bytes(ctx));
  if (e != cudaSuccess) {
    ctx->table = nullptr;
    return cuda_fail(e, "fast-MLS table allocation");
  }
  const int slot = timer_begin(ctx, "fast_table", s);
  e = launch_fast_table(ctx, s);
  timer_end(ctx, slot, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(ctx->table);
    ctx->table = nullptr;
    return cuda_fail(e, "fast-MLS table build");
  }
  return MLS_OK;
}

// The build of mls_build_transfer; with u (and U) also the interpolation of
// mls_interpolate, fused into the exact linear-basis build kernel.
static int build_impl(mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M, int32_t method,
                      void* stream, const void* u, void* U, const void* Vb = nullptr, double dt = 0.0,
                      void* F = nullptr, void* f = nullptr) {
  if (!ctx || !T) return invalid("mls_build_transfer: NULL handle");
  if (T->ctx != ctx) return invalid("mls_build_transfer: transfer belongs to another context");
  if (M < 0) return invalid("mls_build_transfer: negative M");
  if (M > T->cap) {
    set_error("mls_build_transfer: M exceeds the transfer capacity");
    return MLS_ERR_CAPACITY;
  }
  if (method != MLS_EXACT && method != MLS_FAST && method != MLS_SURROGATE)
    return invalid("mls_build_transfer: unknown method");
  if (method == MLS_SURROGATE && (!ctx->mlp_pack || ctx->opt.real != MLS_F32 || ctx->opt.basis != 4)) {
    set_error("mls_build_transfer: the surrogate needs a single-precision, linear-basis context with trained or "
              "loaded parameters");
    return MLS_ERR_UNSUPPORTED;
  }
  if (M > 0 && (!x || !area)) return invalid("mls_build_transfer: NULL marker arrays");
  cudaStream_t s = (cudaStream_t)stream;
  if (method == MLS_FAST) {
    int rc = ensure_table(ctx, s);
    if (rc != MLS_OK) return rc;
  }
  T->M = M;
  T->method = method;
  // Markers that mls_marker_prep_locate has already located, all of them, in
  // these arrays: the counters, bins and tile keys are in place.
  const bool located = M > 0 && T->pre_M == M && T->pre_done == M && T->pre_x == x && T->pre_area == area;
  T->pre_M = -1;
  cudaError_t e;
  int slot = -1;
  if (!located) {
    if ((e = cudaMemsetAsync(T->status, 0, 4 * sizeof(unsigned long long), s)) != cudaSuccess)
      return cuda_fail(e, "mls_build_transfer: status reset");
    if (M == 0) return MLS_OK;
    slot = timer_begin(ctx, "bin_reset", s);
    e = cudaMemsetAsync(T->counts, 0, (size_t)ctx->tiles.nbins * 4, s);
    timer_end(ctx, slot, s);
    if (e != cudaSuccess) return cuda_fail(e, "mls_build_transfer: bin reset");
    slot = timer_begin(ctx, "locate", s);
    e = launch_locate(ctx, T, x, area, M, s);
    timer_end(ctx, slot, s);
    if (e != cudaSuccess) return cuda_fail(e, "mls_build_transfer: locate");
  }
  e = launch_scan(T, ctx->tiles.nbins, s, ctx);
  if (e != cudaSuccess) return cuda_fail(e, "mls_build_transfer: scan");
  slot = timer_begin(ctx, "scatter", s);
  e = launch_scatter(ctx, T, M, s);
  timer_end(ctx, slot, s);
  if (e != cudaSuccess) return cuda_fail(e, "mls_build_transfer: scatter");
  slot = timer_begin(ctx, "tile_sort", s);
  e = launch_tile_sort(ctx, T, M, s);
  timer_end(ctx, slot, s);
  if (e != cudaSuccess) return cuda_fail(e, "mls_build_transfer: tile sort");
  if (u && method == MLS_EXACT && ctx->opt.basis == 4) {
    slot = timer_begin(ctx, F ? "build_exact_forcing" : "build_exact_interp", s);
    e = launch_build_exact_interp(ctx, T, x, area, M, u, U, s, Vb, dt, F);
    timer_end(ctx, slot, s);
    if (e != cudaSuccess) return cuda_fail(e, "mls_build_interpolate: build");
    if (F) {
      slot = timer_begin(ctx, "spread", s);
      e = launch_spread(ctx, T, F, f, s);
      timer_end(ctx, slot, s);
      if (e != cudaSuccess) return cuda_fail(e, "mls_build_direct_forcing: spread");
    }
    return MLS_OK;
  }
  slot = timer_begin(ctx, method == MLS_EXACT ? "build_exact" : method == MLS_FAST ? "build_fast" : "build_surrogate",
                     s);
  e = method == MLS_EXACT  ? launch_build_exact(ctx, T, x, area, M, s)
      : method == MLS_FAST ? launch_build_fast(ctx, T, x, area, M, s)
                           : launch_build_surrogate(ctx, T, x, area, M, s);
  timer_end(ctx, slot, s);
  if (e != cudaSuccess) return cuda_fail(e, "mls_build_transfer: build");
  if (F) {
    slot = timer_begin(ctx, "direct_forcing", s);
    e = launch_direct_forcing(ctx, T, u, Vb, dt, U, F, f, s);
    timer_end(ctx, slot, s);
    if (e != cudaSuccess) return cuda_fail(e, "mls_build_direct_forcing: direct forcing");
  } else if (u) {
    slot = timer_begin(ctx, "interp", s);
    e = launch_interp(ctx, T, u, U, s);
    timer_end(ctx, slot, s);
    if (e != cudaSuccess) return cuda_fail(e, "mls_build_interpolate: interpolation");
  }
  return MLS_OK;
}

int mls_build_transfer(mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M, int32_t method,
                       void* stream) {
  return build_impl(ctx, T, x, area, M, method, stream, nullptr, nullptr);
}

int mls_build_direct_forcing(mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M,
                             int32_t method, const void* u, const void* Vb, double dt, void* U, void* F, void* f,
                             void* stream) {
  if (!(dt > 0.0) || !std::isfinite(dt)) return invalid("mls_build_direct_forcing: dt must be positive and finite");
  if (M > 0 && (!u || !Vb || !F || !f)) return invalid("mls_build_direct_forcing: NULL field, velocity or force");
  if (M == 0) return build_impl(ctx, T, x, area, M, method, stream, nullptr, nullptr);
  return build_impl(ctx, T, x, area, M, method, stream, u, U, Vb, dt, F, f);
}

int mls_build_interpolate(mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M, int32_t method,
                          const void* u, void* U, void* stream) {
  if (M > 0 && (!u || !U)) return invalid("mls_build_interpolate: NULL field or output");
  if (M == 0) return build_impl(ctx, T, x, area, M, method, stream, nullptr, nullptr);
  return build_impl(ctx, T, x, area, M, method, stream, u, U);
}

int mls_interpolate(mls_ctx* ctx, const mls_transfer* T, const void* u, void* U, void* stream) {
  if (!ctx || !T) return invalid("mls_interpolate: NULL handle");
  if (T->ctx != ctx) return invalid("mls_interpolate: transfer belongs to another context");
  if (T->M > 0 && (!u || !U)) return invalid("mls_interpolate: NULL field or output");
  cudaStream_t s = (cudaStream_t)stream;
  const int slot = timer_begin(ctx, "interp", s);
  cudaError_t e = launch_interp(ctx, T, u, U, s);
  timer_end(ctx, slot, s);
  if (e != cudaSuccess) return cuda_fail(e, "mls_interpolate");
  return MLS_OK;
}

int mls_interpolate_gradient(mls_ctx* ctx, const mls_transfer* T, const void* x, const void* u, void* G,
                             void* stream) {
  if (!ctx || !T) return invalid("mls_interpolate_gradient: NULL handle");
  if (T->ctx != ctx) return invalid("mls_interpolate_gradient: transfer belongs to another context");
  if (T->M > 0 && (!x || !u || !G)) return invalid("mls_interpolate_gradient: NULL positions, field or output");
  if (ctx->opt.basis != 4) {
    set_error("mls_interpolate_gradient: derivative shape functions are implemented for the linear basis only");
    return MLS_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int slot = timer_begin(ctx, "interp_gradient", s);
  cudaError_t e = launch_interp_gradient(ctx, T, x, u, G, s);
  timer_end(ctx, slot, s);
  if (e != cudaSuccess) return cuda_fail(e, "mls_interpolate_gradient");
  return MLS_OK;
}

int mls_spread(mls_ctx* ctx, const mls_transfer* T, const void* F, void* f, void* stream) {
  if (!ctx || !T) return invalid("mls_spread: NULL handle");
  if (T->ctx != ctx) return invalid("mls_spread: transfer belongs to another context");
  if (T->M > 0 && (!F || !f)) return invalid("mls_spread: NULL forces or field");
  cudaStream_t s = (cudaStream_t)stream;
  const int slot = timer_begin(ctx, "spread", s);
  cudaError_t e = launch_spread(ctx, T, F, f, s);
  timer_end(ctx, slot, s);
  if (e != cudaSuccess) return cuda_fail(e, "mls_spread");
  return MLS_OK;
}

int mls_direct_forcing(mls_ctx* ctx, const mls_transfer* T, const void* u, const void* Vb, double dt, void* U,
                       void* F, void* f, void* stream) {
  if (!ctx || !T) return invalid("mls_direct_forcing: NULL handle");
  if (T->ctx != ctx) return invalid("mls_direct_forcing: transfer belongs to another context");
  if (!(dt > 0.0) || !std::isfinite(dt)) return invalid("mls_direct_forcing: dt must be positive and finite");
  if (T->M > 0 && (!u || !Vb || !F || !f)) return invalid("mls_direct_forcing: NULL field, velocity or force");
  cudaStream_t s = (cudaStream_t)stream;
  const int slot = timer_begin(ctx, "direct_forcing", s);
  cudaError_t e = launch_direct_forcing(ctx, T, u, Vb, dt, U, F, f, s);
  timer_end(ctx, slot, s);
  if (e != cudaSuccess) return cuda_fail(e, "mls_direct_forcing");
  return MLS_OK;
}

int mls_collisions(mls_ctx* ctx, const mls_transfer* T, const int32_t* body, int32_t* flag, int32_t* coll,
                   unsigned long long* n_colliding, void* stream) {
  if (!ctx || !T) return invalid("mls_collisions: NULL handle");
  if (T->ctx != ctx) return invalid("mls_collisions: transfer belongs to another context");
  if (T->M > 0 && (!body || !flag)) return invalid("mls_collisions: NULL body or flag array");
  cudaStream_t s = (cudaStream_t)stream;
  const int slot = timer_begin(ctx, "collisions", s);
  cudaError_t e = launch_collisions(ctx, T, body, flag, coll, n_colliding, s);
  timer_end(ctx, slot, s);
  if (e != cudaSuccess) return cuda_fail(e, "mls_collisions");
  return MLS_OK;
}

int mls_transfer_view(const mls_transfer* T, mls_transfer_arrays* out) {
  if (!T || !out) return invalid("mls_transfer_view: NULL argument");
  out->M = T->M;
  out->phi = T->phi;
  out->c = T->c;
  out->home = T->home;
  out->perm = T->perm;
  out->capacity = T->cap;
  return MLS_OK;
}

int mls_transfer_status(const mls_transfer* T, void* stream, mls_status* out) {
  if (!T || !out) return invalid("mls_transfer_status: NULL argument");
  unsigned long long h[4] = {0, 0, 0, 0};
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(h, T->status, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "mls_transfer_status");
  out->dropped = (int64_t)h[0];
  out->nonfinite = (int64_t)h[1];
  out->refined_fp64 = (int64_t)h[2];
  out->surrogate_fallback = (int64_t)h[3];
  if (h[0] > 0) {
    set_error("some markers were dropped");
    return MLS_ERR_OUT_OF_DOMAIN;
  }
  return MLS_OK;
}

int mls_fast_table(mls_ctx* ctx, void* stream, const void** table, int64_t* n_classes, int32_t* n_sub) {
  if (!ctx || !table || !n_classes || !n_sub) return invalid("mls_fast_table: NULL argument");
  int rc = ensure_table(ctx, (cudaStream_t)stream);
  if (rc != MLS_OK) return rc;
  *table = ctx->table;
  *n_classes = ctx->n_classes;
  *n_sub = ctx->opt.n_sub;
  return MLS_OK;
}

int mls_timing_enable(mls_ctx* ctx, int32_t on) {
  if (!ctx) return invalid("mls_timing_enable: NULL ctx");
  ctx->timing = on ? 1 : 0;
  return MLS_OK;
}

int mls_timing_read(mls_ctx* ctx, mls_kernel_time* out, int32_t max, int32_t* n) {
  if (!ctx || !n || (max > 0 && !out)) return invalid("mls_timing_read: NULL argument");
  for (size_t q = 0; q < ctx->events_used; ++q) {
    mls_event_pair& p = ctx->events[q];
    cudaError_t e = cudaEventSynchronize(p.stop);
    if (e != cudaSuccess) return cuda_fail(e, "mls_timing_read");
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, p.start, p.stop);
    if (e != cudaSuccess) return cuda_fail(e, "mls_timing_read");
    ctx->timers[p.timer].launches += 1;
    ctx->timers[p.timer].total_ms += ms;
  }
  ctx->events_used = 0;
  int32_t k = 0;
  for (size_t q = 0; q < ctx->timers.size() && k < max; ++q) {
    out[k].name = ctx->timers[q].name;
    out[k].launches = ctx->timers[q].launches;
    out[k].total_ms = ctx->timers[q].total_ms;
    ++k;
  }
  *n = k;
  for (auto& t : ctx->timers) {
    t.launches = 0;
    t.total_ms = 0.0;
  }
  return MLS_OK;
}

}  // extern "C"
