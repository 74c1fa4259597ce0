// Checkpoint and resume of a context's precomputed state: the fast-MLS table
// (Section 2, Fig. 1b/1c: shape functions at the n_sub^3 sub-Eulerian points,
// one class per cell of the non-uniform axis) and the surrogate's float32
// parameters.  Neither depends on the markers, so a run that restarts on the
// same grid reloads them instead of rebuilding or retraining.
//
// File layout (native byte order; both targets are little-endian):
//   char     magic[8]   "MLSCKPT\0"
//   uint32   version    1
//   uint32   flags      bit 0: table present, bit 1: surrogate present
//   uint64   key        FNV-1a 64 over the grid and options the state depends on
//   [table]  int32 class_axis, int32 n_sub, int64 n_classes, uint64 bytes, bytes of data
//   [surrogate] uint64 count (= MLS_MLP_PARAMS), count float32 values
//   uint64   check      FNV-1a 64 over every preceding byte
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mls_host.h"

using namespace mls;

namespace {

constexpr char kMagic[8] = {'M', 'L', 'S', 'C', 'K', 'P', 'T', '\0'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kHasTable = 1u, kHasSurrogate = 2u;

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  }
  template <typename T> void put(const T& v) { add(&v, sizeof(T)); }
};

// Everything the table and the surrogate are a function of: the grid (face
// coordinates, periodicity), the Gaussian width eps, the sub-point count, the
// basis size and the arithmetic precision.
uint64_t context_key(const mls_ctx* ctx) {
  Fnv f;
  for (int d = 0; d < 3; ++d) {
    f.put<int32_t>(ctx->n[d]);
    f.put<int32_t>(ctx->periodic[d]);
  }
  f.put<int32_t>(ctx->opt.real);
  f.put<int32_t>(ctx->opt.n_sub);
  f.put<int32_t>(ctx->opt.basis);
  f.put<double>(ctx->opt.eps);
  for (int d = 0; d < 3; ++d) f.add(ctx->faces_host[d].data(), ctx->faces_host[d].size() * sizeof(double));
  return f.h;
}

struct Writer {
  std::vector<unsigned char> buf;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    buf.insert(buf.end(), b, b + n);
  }
  template <typename T> void put(const T& v) { add(&v, sizeof(T)); }
};

struct Reader {
  const unsigned char* p;
  size_t n, at = 0;
  bool take(void* dst, size_t k) {
    if (k > n - at) return false;
    std::memcpy(dst, p + at, k);
    at += k;
    return true;
  }
  template <typename T> bool get(T* v) { return take(v, sizeof(T)); }
};

int bad_file(const char* what) {
  set_error(std::string("mls_load: ") + what);
  return MLS_ERR_INVALID_ARG;
}

}  // namespace

int mls_save(mls_ctx* ctx, const char* path) {
  if (!ctx || !path) {
    set_error("mls_save: NULL argument");
    return MLS_ERR_INVALID_ARG;
  }
  // Tables and parameters are written by earlier launches on any stream.
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "mls_save");
  Writer w;
  w.add(kMagic, sizeof(kMagic));
  w.put<uint32_t>(kVersion);
  const uint32_t flags = (ctx->table ? kHasTable : 0u) | (ctx->mlp_theta ? kHasSurrogate : 0u);
  w.put<uint32_t>(flags);
  w.put<uint64_t>(context_key(ctx));
  if (ctx->table) {
    const uint64_t bytes = fast_table_bytes(ctx);
    w.put<int32_t>(ctx->class_axis);
    w.put<int32_t>(ctx->opt.n_sub);
    w.put<int64_t>(ctx->n_classes);
    w.put<uint64_t>(bytes);
    const size_t at = w.buf.size();
    w.buf.resize(at + bytes);
    if ((e = cudaMemcpy(w.buf.data() + at, ctx->table, bytes, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "mls_save: table copy");
  }
  if (ctx->mlp_theta) {
    w.put<uint64_t>((uint64_t)MLS_MLP_PARAMS);
    const size_t at = w.buf.size();
    w.buf.resize(at + MLS_MLP_PARAMS * sizeof(float));
    if ((e = cudaMemcpy(w.buf.data() + at, ctx->mlp_theta, MLS_MLP_PARAMS * sizeof(float),
                        cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "mls_save: surrogate copy");
  }
  Fnv check;
  check.add(w.buf.data(), w.buf.size());
  w.put<uint64_t>(check.h);
  // Write beside the target and rename, so a crash never leaves a torn file
  // under the checkpoint's name.
  const std::string tmp = std::string(path) + ".partial";
  FILE* fp = std::fopen(tmp.c_str(), "wb");
  if (!fp) {
    set_error("mls_save: cannot open " + tmp);
    return MLS_ERR_INVALID_ARG;
  }
  const bool ok = std::fwrite(w.buf.data(), 1, w.buf.size(), fp) == w.buf.size();
  const bool closed = std::fclose(fp) == 0;
  if (!ok || !closed || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    set_error(std::string("mls_save: cannot write ") + path);
    return MLS_ERR_INVALID_ARG;
  }
  return MLS_OK;
}

int mls_load(mls_ctx* ctx, const char* path) {
  if (!ctx || !path) {
    set_error("mls_load: NULL argument");
    return MLS_ERR_INVALID_ARG;
  }
  std::vector<unsigned char> buf;
  {
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return bad_file("cannot open the file");
    unsigned char chunk[1 << 16];
    size_t k;
    while ((k = std::fread(chunk, 1, sizeof(chunk), fp)) > 0) buf.insert(buf.end(), chunk, chunk + k);
    const bool err = std::ferror(fp) != 0;
    std::fclose(fp);
    if (err) return bad_file("read error");
  }
  if (buf.size() < sizeof(kMagic) + 16 + 8) return bad_file("file too short");
  uint64_t stored_check;
  std::memcpy(&stored_check, buf.data() + buf.size() - 8, 8);
  Fnv check;
  check.add(buf.data(), buf.size() - 8);
  if (std::memcmp(buf.data(), kMagic, sizeof(kMagic)) != 0) return bad_file("not a checkpoint (magic)");
  if (check.h != stored_check) return bad_file("checksum mismatch (truncated or corrupt)");
  Reader r{buf.data(), buf.size() - 8, sizeof(kMagic)};
  uint32_t version, flags;
  uint64_t key;
  r.get(&version);
  r.get(&flags);
  r.get(&key);
  if (version != kVersion) return bad_file("unsupported version");
  if (flags & ~(kHasTable | kHasSurrogate)) return bad_file("unknown flags");
  if (key != context_key(ctx)) return bad_file("written for another grid or option set");

  // Parse and validate everything before touching the context.
  const unsigned char* table_data = nullptr;
  uint64_t table_bytes = 0;
  if (flags & kHasTable) {
    int32_t axis, n_sub;
    int64_t n_classes;
    if (!r.get(&axis) || !r.get(&n_sub) || !r.get(&n_classes) || !r.get(&table_bytes))
      return bad_file("truncated table header");
    int rc = fast_table_layout(ctx);
    if (rc != MLS_OK) return rc;
    if (axis != ctx->class_axis || n_sub != ctx->opt.n_sub || n_classes != ctx->n_classes ||
        table_bytes != fast_table_bytes(ctx))
      return bad_file("table shape does not match the context");
    if (table_bytes > r.n - r.at) return bad_file("truncated table");
    table_data = r.p + r.at;
    r.at += table_bytes;
  }
  std::vector<float> theta;
  if (flags & kHasSurrogate) {
    uint64_t count;
    if (!r.get(&count) || count != (uint64_t)MLS_MLP_PARAMS) return bad_file("bad surrogate parameter count");
    theta.resize(MLS_MLP_PARAMS);
    if (!r.take(theta.data(), theta.size() * sizeof(float))) return bad_file("truncated surrogate parameters");
  }
  if (r.at != r.n) return bad_file("trailing bytes");
  // The surrogate part needs a context that can hold it: checked before the
  // table is touched, so a refusal leaves the context as it was.
  if (!theta.empty()) {
    int rc = surrogate_check(ctx, "mls_load");
    if (rc != MLS_OK) return rc;
  }

  cudaError_t e;
  if (table_data) {
    const bool fresh = !ctx->table;
    if (fresh && (e = cudaMalloc(&ctx->table, table_bytes)) != cudaSuccess) {
      ctx->table = nullptr;
      return cuda_fail(e, "mls_load: table allocation");
    }
    // A table in use by launches still in flight is replaced only after they end.
    if ((e = cudaDeviceSynchronize()) != cudaSuccess ||
        (e = cudaMemcpy(ctx->table, table_data, table_bytes, cudaMemcpyHostToDevice)) != cudaSuccess) {
      // A table allocated here never holds partial contents: later fast builds
      // rebuild it instead.
      if (fresh) {
        cudaFree(ctx->table);
        ctx->table = nullptr;
      }
      return cuda_fail(e, "mls_load: table copy");
    }
  }
  if (!theta.empty()) {
    int rc = mls_surrogate_params(ctx, theta.data(), MLS_MLP_PARAMS, 1);
    if (rc != MLS_OK) return rc;
  }
  return MLS_OK;
}
