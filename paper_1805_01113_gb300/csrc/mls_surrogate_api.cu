// C ABI of the learned surrogate (training, parameters, test entry points).
#include <cmath>
#include <vector>

#include "mls_host.h"

using namespace mls;

namespace {

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

int need_surrogate_grid(mls_ctx* ctx, const char* who) {
  if (ctx->opt.real != MLS_F32)
    return fail(MLS_ERR_UNSUPPORTED, std::string(who) + ": the surrogate runs in single-precision contexts");
  if (ctx->opt.basis != 4)
    return fail(MLS_ERR_UNSUPPORTED, std::string(who) + ": the surrogate learns linear-basis shape functions");
  if (surrogate_class_axis(ctx) == -2)
    return fail(MLS_ERR_UNSUPPORTED, std::string(who) + ": the surrogate needs at most one non-uniform axis");
  return MLS_OK;
}

int ensure_params(mls_ctx* ctx) {
  cudaError_t e;
  if (!ctx->mlp_theta && (e = cudaMalloc(&ctx->mlp_theta, MLS_MLP_PARAMS * sizeof(float))) != cudaSuccess) {
    ctx->mlp_theta = nullptr;
    return cuda_fail(e, "surrogate parameter allocation");
  }
  if (!ctx->mlp_pack && (e = cudaMalloc(&ctx->mlp_pack, mlp_pack_bytes())) != cudaSuccess) {
    ctx->mlp_pack = nullptr;
    return cuda_fail(e, "surrogate weight allocation");
  }
  return MLS_OK;
}

// Device allocations freed when the scope ends.
struct Scratch {
  std::vector<void*> p;
  cudaError_t alloc(void** out, size_t bytes) {
    cudaError_t e = cudaMalloc(out, bytes);
    if (e == cudaSuccess) p.push_back(*out);
    return e;
  }
  ~Scratch() {
    for (void* q : p) cudaFree(q);
  }
};

}  // namespace

namespace mls {
int surrogate_check(mls_ctx* ctx, const char* who) { return need_surrogate_grid(ctx, who); }
}  // namespace mls

extern "C" {

int mls_train_options_default(mls_train_options* o) {
  if (!o) return fail(MLS_ERR_INVALID_ARG, "mls_train_options_default: NULL");
  o->n_samples = 1 << 20;
  o->epochs = 128;
  o->batch = 1024;
  o->lr = 3e-3;
  o->lr_final = 1e-6;
  o->seed = 1805011135ULL;
  return MLS_OK;
}

int mls_surrogate_train(mls_ctx* ctx, const mls_train_options* o_in, void* stream, double* loss) {
  if (!ctx) return fail(MLS_ERR_INVALID_ARG, "mls_surrogate_train: NULL context");
  mls_train_options o;
  if (o_in) o = *o_in; else mls_train_options_default(&o);
  if (o.n_samples < 1 || o.n_samples > (int64_t(1) << 26) || o.epochs < 1 || o.batch < 128 || o.batch > 65536 ||
      o.batch % 128 != 0 || !(o.lr > 0) || !(o.lr_final > 0))
    return fail(MLS_ERR_INVALID_ARG, "mls_surrogate_train: bad options");
  int rc = need_surrogate_grid(ctx, "mls_surrogate_train");
  if (rc != MLS_OK) return rc;
  if ((rc = ensure_params(ctx)) != MLS_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch w;
  float *X, *T, *work, *grad, *m, *v, *lsum;
  cudaError_t e;
  if ((e = w.alloc((void**)&X, (size_t)o.n_samples * 6 * 4)) != cudaSuccess ||
      (e = w.alloc((void**)&T, (size_t)o.n_samples * 27 * 4)) != cudaSuccess ||
      (e = w.alloc((void**)&work, mlp_train_floats(o.batch) * 4)) != cudaSuccess ||
      (e = w.alloc((void**)&grad, MLS_MLP_PARAMS * 4)) != cudaSuccess ||
      (e = w.alloc((void**)&m, MLS_MLP_PARAMS * 4)) != cudaSuccess ||
      (e = w.alloc((void**)&v, MLS_MLP_PARAMS * 4)) != cudaSuccess ||
      (e = w.alloc((void**)&lsum, 4)) != cudaSuccess)
    return cuda_fail(e, "mls_surrogate_train: workspace");
  std::vector<float> theta0(MLS_MLP_PARAMS);
  mlp_init_params(o.seed, theta0.data());
  if ((e = cudaMemcpy(ctx->mlp_theta, theta0.data(), MLS_MLP_PARAMS * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemsetAsync(m, 0, MLS_MLP_PARAMS * 4, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(v, 0, MLS_MLP_PARAMS * 4, s)) != cudaSuccess ||
      (e = launch_mlp_samples(ctx, 0, o.n_samples, o.seed, X, T, s)) != cudaSuccess)
    return cuda_fail(e, "mls_surrogate_train: set-up");
  const int64_t per_epoch = (o.n_samples + o.batch - 1) / o.batch;
  const int64_t total = per_epoch * o.epochs;
  const uint64_t batch_seed = o.seed ^ 0x6D6C732D62617463ULL;
  double bc1 = 1.0, bc2 = 1.0;
  const int slot = timer_begin(ctx, "surrogate_train", s);
  for (int64_t step = 0; step < total; ++step) {
    if (step == total - per_epoch && (e = cudaMemsetAsync(lsum, 0, 4, s)) != cudaSuccess) break;
    const double frac = (double)step / (double)total;
    const double lr = o.lr_final + 0.5 * (o.lr - o.lr_final) * (1.0 + std::cos(M_PI * frac));
    bc1 *= 0.9;
    bc2 *= 0.999;
    if ((e = launch_mlp_grad(ctx->mlp_theta, X, T, o.n_samples, o.batch, true, (uint64_t)step * o.batch,
                             batch_seed, work, grad, lsum, s)) != cudaSuccess)
      break;
    if ((e = launch_adam(ctx->mlp_theta, grad, m, v, (float)lr, (float)(1.0 - bc1), (float)(1.0 - bc2), s)) !=
        cudaSuccess)
      break;
  }
  timer_end(ctx, slot, s);
  if (e == cudaSuccess) e = launch_mlp_pack(ctx->mlp_theta, ctx->mlp_pack, s);
  float l = 0.f;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&l, lsum, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "mls_surrogate_train");
  if (loss) *loss = (double)l / ((double)per_epoch * o.batch * 27.0);
  return MLS_OK;
}

int mls_surrogate_params(mls_ctx* ctx, float* host, int64_t n, int32_t set) {
  if (!ctx || !host) return fail(MLS_ERR_INVALID_ARG, "mls_surrogate_params: NULL argument");
  if (n != MLS_MLP_PARAMS) return fail(MLS_ERR_INVALID_ARG, "mls_surrogate_params: n must be MLS_MLP_PARAMS");
  cudaError_t e;
  if (set) {
    int rc = need_surrogate_grid(ctx, "mls_surrogate_params");
    if (rc != MLS_OK) return rc;
    if ((rc = ensure_params(ctx)) != MLS_OK) return rc;
    if ((e = cudaMemcpy(ctx->mlp_theta, host, n * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = launch_mlp_pack(ctx->mlp_theta, ctx->mlp_pack, 0)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess)
      return cuda_fail(e, "mls_surrogate_params");
    return MLS_OK;
  }
  if (!ctx->mlp_theta) return fail(MLS_ERR_UNSUPPORTED, "mls_surrogate_params: no parameters yet");
  if ((e = cudaMemcpy(host, ctx->mlp_theta, n * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "mls_surrogate_params");
  return MLS_OK;
}

int mls_surrogate_samples(mls_ctx* ctx, int64_t first, int64_t count, uint64_t seed, float* X, float* T,
                          void* stream) {
  if (!ctx || (count > 0 && (!X || !T)) || first < 0 || count < 0)
    return fail(MLS_ERR_INVALID_ARG, "mls_surrogate_samples: bad argument");
  int rc = need_surrogate_grid(ctx, "mls_surrogate_samples");
  if (rc != MLS_OK) return rc;
  cudaError_t e = launch_mlp_samples(ctx, first, count, seed, X, T, (cudaStream_t)stream);
  return e == cudaSuccess ? MLS_OK : cuda_fail(e, "mls_surrogate_samples");
}

int mls_surrogate_forward(mls_ctx* ctx, const float* X, int32_t B, int32_t mode, float* Y, void* stream) {
  if (!ctx || B < 0 || (B > 0 && (!X || !Y)) || (mode != MLS_F32 && mode != MLS_BF16))
    return fail(MLS_ERR_INVALID_ARG, "mls_surrogate_forward: bad argument");
  if (!ctx->mlp_theta) return fail(MLS_ERR_UNSUPPORTED, "mls_surrogate_forward: no parameters yet");
  if (B == 0) return MLS_OK;
  cudaError_t e = launch_mlp_forward(ctx->mlp_theta, ctx->mlp_pack, X, B, mode, Y, (cudaStream_t)stream);
  return e == cudaSuccess ? MLS_OK : cuda_fail(e, "mls_surrogate_forward");
}

int mls_surrogate_loss_grad(mls_ctx* ctx, const float* X, const float* T, int32_t B, float* grad, float* loss,
                            void* stream) {
  if (!ctx || B <= 0 || B % 128 != 0 || !X || !T || !grad || !loss)
    return fail(MLS_ERR_INVALID_ARG, "mls_surrogate_loss_grad: bad argument");
  if (!ctx->mlp_theta) return fail(MLS_ERR_UNSUPPORTED, "mls_surrogate_loss_grad: no parameters yet");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch w;
  float* work;
  cudaError_t e = w.alloc((void**)&work, mlp_train_floats(B) * 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, 4, s);
  if (e == cudaSuccess) e = launch_mlp_grad(ctx->mlp_theta, X, T, B, B, false, 0, 0, work, grad, loss, s);
  if (e == cudaSuccess) e = launch_scale1(loss, 1.f / (27.f * (float)B), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? MLS_OK : cuda_fail(e, "mls_surrogate_loss_grad");
}

}  // extern "C"
