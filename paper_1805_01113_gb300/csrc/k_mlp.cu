// Learned surrogate of exact-MLS: training-set generation, float32
// forward/backward and Adam kernels, and the bfloat16 tensor-core network
// used by MLS_SURROGATE builds (projection onto linear reproduction, exact
// fallback).
#include <algorithm>
#include <cmath>

#include "mls_host.h"

namespace mls {

// Flat parameter layout: W1[64][6], b1[64], W2[64][64], b2[64], W3[27][64], b3[27].
constexpr int kIn = 6, kH = 64, kOut = 27;
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kOut * kH, kParams = ob3 + kOut;
static_assert(kParams == MLS_MLP_PARAMS, "parameter count");
constexpr int kMlpThreads = 128;

// ---- counter-based draws: the splitmix64 output function --------------------
__host__ __device__ inline uint64_t splitmix64(uint64_t counter, uint64_t seed) {
  uint64_t z = seed + (counter + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__host__ __device__ inline double uniform01(uint64_t counter, uint64_t seed) {
  return (double)(splitmix64(counter, seed) >> 40) * (1.0 / 16777216.0);
}

void mlp_init_params(uint64_t seed, float* theta) {
  for (int q = 0; q < kParams; ++q) theta[q] = 0.f;
  struct Block { int off, fo, fi; } W[3] = {{oW1, kH, kIn}, {oW2, kH, kH}, {oW3, kOut, kH}};
  for (const Block& b : W) {
    const double a = std::sqrt(6.0 / (b.fi + b.fo));
    for (int q = 0; q < b.fo * b.fi; ++q)
      theta[b.off + q] = (float)((2.0 * uniform01((uint64_t)(b.off + q), seed) - 1.0) * a);
  }
}

// Features of the surrogate from the node geometry of the non-uniform axis.
struct SurrogateAxes {
  int c;          // class axis (non-uniform, or 2 when all are uniform)
  int u;          // first other axis
};

// ---- training points -----------------------------------------------------------
// Sample s: offsets t_d = u(4s+d) - 1/2, home index along the class axis from
// draw 4s+3; label = exact-MLS phi in double (Eqs. 3-6), rounded to float.
__global__ void k_mlp_samples(Grid<double> gd, SurrogateAxes ax, int lo, int span, int64_t first, int64_t count,
                              uint64_t seed, double inv_eps2, float* __restrict__ X, float* __restrict__ T) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const uint64_t s = (uint64_t)(first + q);
  double t[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) t[d] = uniform01(4 * s + d, seed) - 0.5;
  const uint64_t z = splitmix64(4 * s + 3, seed);
  const int cls = lo + (int)(((z >> 32) * (uint64_t)span) >> 32);
  AxisNodes<double> nd[3];
  double wm_c = 1, wh_c = 1, wp_c = 1;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const Axis<double>& a = gd.ax[d];
    const int i = d == ax.c ? cls : a.n / 2;
    const double wm = width_of(a, wrap(i - 1, a.n, a.periodic)), wh = width_of(a, i),
                 wp = width_of(a, wrap(i + 1, a.n, a.periodic));
    nd[d] = axis_nodes_at(t[d], wm, wh, wp);
    if (d == ax.c) {
      wm_c = wm;
      wh_c = wh;
      wp_c = wp;
    }
  }
  const double wu = width_of(gd.ax[ax.u], gd.ax[ax.u].n / 2);
  float* x = X + q * kIn;
  x[0] = (float)t[0];
  x[1] = (float)t[1];
  x[2] = (float)t[2];
  x[3] = (float)log(wm_c / wh_c);
  x[4] = (float)log(wp_c / wh_c);
  x[5] = (float)log(wh_c / wu);
  double phi[27];
  if (!shape_exact<double>(nd, inv_eps2, 0, phi, nullptr))
    for (int k = 0; k < 27; ++k) phi[k] = 0.0;
  for (int k = 0; k < 27; ++k) T[q * kOut + k] = (float)phi[k];
}

// ---- float32 training path -------------------------------------------------------
// One sample per thread.  Activations are kept feature-major ([feature][batch])
// so the per-thread writes and the weight-gradient reads are coalesced.
struct TrainBuffers {
  float* Xb;    // [6][B]
  float* H1;    // [64][B]
  float* H2;    // [64][B]
  float* dY;    // [27][B]
  float* dZ1;   // [64][B]
  float* dZ2;   // [64][B]
};

__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// Forward (and with BWD the backward deltas) of the float32 network for a
// minibatch.  With GATHER the batch is drawn from the training set
// (index = splitmix64 draw mod n); otherwise sample b is row b of Xin/Tin.
template <bool BWD, bool GATHER>
__global__ void __launch_bounds__(kMlpThreads) k_mlp_fwd(const float* __restrict__ theta, const float* __restrict__ Xin,
                                                         const float* __restrict__ Tin, int64_t n_all, int B,
                                                         uint64_t draw_base, uint64_t seed, TrainBuffers tb,
                                                         float* __restrict__ Yout, float* __restrict__ loss_sum) {
  extern __shared__ float sm[];
  float* W = sm;                                   // kParams
  float* h1 = W + kParams + 1;                     // [64][128]
  float* h2 = h1 + kH * kMlpThreads;               // [64][128]
  float* yv = h2 + kH * kMlpThreads;               // [27][128]
  __shared__ float red[kMlpThreads / 32];
  const int tid = threadIdx.x;
  for (int q = tid; q < kParams; q += kMlpThreads) W[q] = theta[q];
  __syncthreads();
  const int b = blockIdx.x * kMlpThreads + tid;
  const bool act = b < B;
  int64_t src = b;
  if (GATHER && act) src = (int64_t)((splitmix64(draw_base + (uint64_t)b, seed) >> 11) % (uint64_t)n_all);
  float x[kIn];
#pragma unroll
  for (int i = 0; i < kIn; ++i) x[i] = act ? Xin[src * kIn + i] : 0.f;
  for (int j = 0; j < kH; ++j) {
    float z = W[ob1 + j];
#pragma unroll
    for (int i = 0; i < kIn; ++i) z += W[oW1 + j * kIn + i] * x[i];
    h1[j * kMlpThreads + tid] = tanhf(z);
  }
  for (int j = 0; j < kH; ++j) {
    float z = W[ob2 + j];
    for (int i = 0; i < kH; ++i) z += W[oW2 + j * kH + i] * h1[i * kMlpThreads + tid];
    h2[j * kMlpThreads + tid] = tanhf(z);
  }
  for (int o = 0; o < kOut; ++o) {
    float y = W[ob3 + o];
    for (int i = 0; i < kH; ++i) y += W[oW3 + o * kH + i] * h2[i * kMlpThreads + tid];
    yv[o * kMlpThreads + tid] = y;
    if (!BWD && act) Yout[(int64_t)b * kOut + o] = y;
  }
  if (!BWD) return;
  // dL/dy for L = sum (y - t)^2 / (B * 27).
  float sq = 0.f;
  const float sc = 2.f / (float)(B * kOut);
  for (int o = 0; o < kOut; ++o) {
    const float r = act ? yv[o * kMlpThreads + tid] - Tin[src * kOut + o] : 0.f;
    sq += r * r;
    yv[o * kMlpThreads + tid] = sc * r;
    if (act) tb.dY[(int64_t)o * B + b] = sc * r;
  }
  const float tot = block_sum(sq, red);
  if (tid == 0) atomicAdd(loss_sum, tot);
  // dZ2 = (W3^T dY) * (1 - h2^2), stored over h2 after its value is saved.
  for (int i = 0; i < kH; ++i) {
    float g = 0.f;
    for (int o = 0; o < kOut; ++o) g += W[oW3 + o * kH + i] * yv[o * kMlpThreads + tid];
    const float hv = h2[i * kMlpThreads + tid];
    if (act) tb.H2[(int64_t)i * B + b] = hv;
    const float dz = act ? g * (1.f - hv * hv) : 0.f;
    if (act) tb.dZ2[(int64_t)i * B + b] = dz;
    h2[i * kMlpThreads + tid] = dz;
  }
  // dZ1 = (W2^T dZ2) * (1 - h1^2).
  for (int i = 0; i < kH; ++i) {
    float g = 0.f;
    for (int j = 0; j < kH; ++j) g += W[oW2 + j * kH + i] * h2[j * kMlpThreads + tid];
    const float hv = h1[i * kMlpThreads + tid];
    if (act) {
      tb.H1[(int64_t)i * B + b] = hv;
      tb.dZ1[(int64_t)i * B + b] = g * (1.f - hv * hv);
    }
  }
  if (act)
#pragma unroll
    for (int i = 0; i < kIn; ++i) tb.Xb[(int64_t)i * B + b] = x[i];
}

// Weight gradients: grad[p] += sum over a chunk of the batch of a(b) * c(b),
// with (a, c) = (delta row, activation row) of parameter p (c = 1 for biases).
__global__ void __launch_bounds__(kMlpThreads) k_mlp_wgrad(int B, int chunk, TrainBuffers tb, float* __restrict__ grad) {
  const int p = blockIdx.x * kMlpThreads + threadIdx.x;
  if (p >= kParams) return;
  const float* a;
  const float* c = nullptr;
  if (p < ob1) {
    a = tb.dZ1 + (int64_t)(p / kIn) * B;
    c = tb.Xb + (int64_t)(p % kIn) * B;
  } else if (p < oW2) {
    a = tb.dZ1 + (int64_t)(p - ob1) * B;
  } else if (p < ob2) {
    a = tb.dZ2 + (int64_t)((p - oW2) / kH) * B;
    c = tb.H1 + (int64_t)((p - oW2) % kH) * B;
  } else if (p < oW3) {
    a = tb.dZ2 + (int64_t)(p - ob2) * B;
  } else if (p < ob3) {
    a = tb.dY + (int64_t)((p - oW3) / kH) * B;
    c = tb.H2 + (int64_t)((p - oW3) % kH) * B;
  } else {
    a = tb.dY + (int64_t)(p - ob3) * B;
  }
  const int b0 = blockIdx.y * chunk, b1 = min(B, b0 + chunk);
  float s = 0.f;
  if (c)
    for (int b = b0; b < b1; ++b) s += a[b] * c[b];
  else
    for (int b = b0; b < b1; ++b) s += a[b];
  atomicAdd(&grad[p], s);
}

__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, float lr, float bc1, float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  const float g = grad[p];
  const float mm = 0.9f * m[p] + 0.1f * g;
  const float vv = 0.999f * v[p] + 0.001f * g * g;
  m[p] = mm;
  v[p] = vv;
  theta[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f);
}

// ---- bfloat16 tensor-core network ------------------------------------------------
// Packed inference weights (bf16, rows padded so fragment loads are
// bank-conflict free): W1p[64][24] (input cols 0..5), W2p[64][72], W3p[32][72]
// (rows 27..31 zero), then float biases b1[64], b2[64], b3[32].
constexpr int kW1s = 24, kW2s = 72, kW3s = 72;
constexpr int kPackBf16 = kH * kW1s + kH * kW2s + 32 * kW3s;
constexpr int kPackBytes = kPackBf16 * 2 + (kH + kH + 32) * 4;

__global__ void k_mlp_pack(const float* __restrict__ theta, unsigned char* __restrict__ pack) {
  __nv_bfloat16* w1 = reinterpret_cast<__nv_bfloat16*>(pack);
  __nv_bfloat16* w2 = w1 + kH * kW1s;
  __nv_bfloat16* w3 = w2 + kH * kW2s;
  float* bias = reinterpret_cast<float*>(pack + kPackBf16 * 2);
  for (int q = threadIdx.x; q < kH * kW1s; q += blockDim.x) {
    const int n = q / kW1s, k = q % kW1s;
    w1[q] = __float2bfloat16_rn(k < kIn ? theta[oW1 + n * kIn + k] : 0.f);
  }
  for (int q = threadIdx.x; q < kH * kW2s; q += blockDim.x) {
    const int n = q / kW2s, k = q % kW2s;
    w2[q] = __float2bfloat16_rn(k < kH ? theta[oW2 + n * kH + k] : 0.f);
  }
  for (int q = threadIdx.x; q < 32 * kW3s; q += blockDim.x) {
    const int n = q / kW3s, k = q % kW3s;
    w3[q] = __float2bfloat16_rn(n < kOut && k < kH ? theta[oW3 + n * kH + k] : 0.f);
  }
  for (int q = threadIdx.x; q < kH; q += blockDim.x) {
    bias[q] = theta[ob1 + q];
    bias[kH + q] = theta[ob2 + q];
  }
  for (int q = threadIdx.x; q < 32; q += blockDim.x) bias[2 * kH + q] = q < kOut ? theta[ob3 + q] : 0.f;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One warp evaluates the network for 32 rows: feat[32][8] (float, cols 6, 7
// unused) -> Y[32][33] (float, cols 0..26).  Fragment layouts are those of
// mma.m16n8k16 (row-major A, column-major B): lane = 4 g + t holds rows g and
// g+8 and columns 2t, 2t+1 (+8); a layer's accumulator fragments of two
// adjacent 8-column tiles are the next layer's A fragment of one 16-deep step.
__device__ __forceinline__ void mlp_warp_bf16(const float* feat, float* Y, const unsigned char* pack) {
  const __nv_bfloat16* w1 = reinterpret_cast<const __nv_bfloat16*>(pack);
  const __nv_bfloat16* w2 = w1 + kH * kW1s;
  const __nv_bfloat16* w3 = w2 + kH * kW2s;
  const float* bias = reinterpret_cast<const float*>(pack + kPackBf16 * 2);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int r0 = mt * 16 + g, r1 = r0 + 8;
    uint32_t a[4];
    a[0] = pack_bf16(feat[r0 * 8 + 2 * t], 2 * t + 1 < 8 ? feat[r0 * 8 + 2 * t + 1] : 0.f);
    a[1] = pack_bf16(feat[r1 * 8 + 2 * t], feat[r1 * 8 + 2 * t + 1]);
    a[2] = 0u;
    a[3] = 0u;
    float c1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int col = nt * 8 + 2 * t;
      c1[nt][0] = c1[nt][2] = bias[col];
      c1[nt][1] = c1[nt][3] = bias[col + 1];
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(w1 + (nt * 8 + g) * kW1s + 2 * t);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(w1 + (nt * 8 + g) * kW1s + 2 * t + 8);
      mma_bf16(c1[nt], a, b0, b1);
    }
    uint32_t a2[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      a2[kt][0] = pack_bf16(tanh_fast(c1[2 * kt][0]), tanh_fast(c1[2 * kt][1]));
      a2[kt][1] = pack_bf16(tanh_fast(c1[2 * kt][2]), tanh_fast(c1[2 * kt][3]));
      a2[kt][2] = pack_bf16(tanh_fast(c1[2 * kt + 1][0]), tanh_fast(c1[2 * kt + 1][1]));
      a2[kt][3] = pack_bf16(tanh_fast(c1[2 * kt + 1][2]), tanh_fast(c1[2 * kt + 1][3]));
    }
    float c2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int col = nt * 8 + 2 * t;
      c2[nt][0] = c2[nt][2] = bias[kH + col];
      c2[nt][1] = c2[nt][3] = bias[kH + col + 1];
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) {
        const __nv_bfloat16* wr = w2 + (nt * 8 + g) * kW2s + kt * 16 + 2 * t;
        mma_bf16(c2[nt], a2[kt], *reinterpret_cast<const uint32_t*>(wr), *reinterpret_cast<const uint32_t*>(wr + 8));
      }
    }
    uint32_t a3[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      a3[kt][0] = pack_bf16(tanh_fast(c2[2 * kt][0]), tanh_fast(c2[2 * kt][1]));
      a3[kt][1] = pack_bf16(tanh_fast(c2[2 * kt][2]), tanh_fast(c2[2 * kt][3]));
      a3[kt][2] = pack_bf16(tanh_fast(c2[2 * kt + 1][0]), tanh_fast(c2[2 * kt + 1][1]));
      a3[kt][3] = pack_bf16(tanh_fast(c2[2 * kt + 1][2]), tanh_fast(c2[2 * kt + 1][3]));
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = nt * 8 + 2 * t;
      float c3[4] = {bias[2 * kH + col], bias[2 * kH + col + 1], bias[2 * kH + col], bias[2 * kH + col + 1]};
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) {
        const __nv_bfloat16* wr = w3 + (nt * 8 + g) * kW3s + kt * 16 + 2 * t;
        mma_bf16(c3, a3[kt], *reinterpret_cast<const uint32_t*>(wr), *reinterpret_cast<const uint32_t*>(wr + 8));
      }
      Y[r0 * 33 + col] = c3[0];
      Y[r0 * 33 + col + 1] = c3[1];
      Y[r1 * 33 + col] = c3[2];
      Y[r1 * 33 + col + 1] = c3[3];
    }
  }
}

// Per-block shared memory of the tensor-core kernels: packed weights, then
// per warp feat[32][8] and Y[32][33].
constexpr int kWarpFeat = 32 * 8, kWarpY = 32 * 33;
constexpr int kBf16Smem = kPackBytes + (kMlpThreads / 32) * (kWarpFeat + kWarpY) * 4;

__device__ __forceinline__ void load_pack(unsigned char* dst, const unsigned char* src) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  for (int q = threadIdx.x; q < kPackBytes / 16; q += blockDim.x) d[q] = s[q];
}

__global__ void __launch_bounds__(kMlpThreads) k_mlp_forward_bf16(const unsigned char* __restrict__ pack_g,
                                                                  const float* __restrict__ X, int B,
                                                                  float* __restrict__ Yout) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_pack(smem, pack_g);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* feat = reinterpret_cast<float*>(smem + kPackBytes) + warp * (kWarpFeat + kWarpY);
  float* Y = feat + kWarpFeat;
  const int b = blockIdx.x * kMlpThreads + threadIdx.x;
#pragma unroll
  for (int i = 0; i < 8; ++i) feat[lane * 8 + i] = (b < B && i < kIn) ? X[(int64_t)b * kIn + i] : 0.f;
  __syncthreads();
  mlp_warp_bf16(feat, Y, smem);
  __syncwarp();
  if (b < B)
    for (int o = 0; o < kOut; ++o) Yout[(int64_t)b * kOut + o] = Y[lane * 33 + o];
}

// Build with the surrogate: features -> network -> residual check of the raw
// output (exact-MLS fallback) -> projection onto linear reproduction -> phi,
// c_l, home.
struct SurrogateArgs {
  Grid<float> g;
  SurrogateAxes ax;
  const float* x;
  const float* area;
  const int32_t* perm;
  int64_t M, cap;
  float* phi;
  float* c;
  int32_t* home;
  unsigned long long* status;
  float inv_eps2;
  float residual_max;
  const unsigned char* pack;
};

// One marker per lane; the warp's 32 markers share the network evaluation
// (feat and Y are the warp's own staging buffers, smem holds the weights).
__device__ __forceinline__ void surrogate_marker(const SurrogateArgs& a, int64_t j, float* feat, float* Y,
                                                 const unsigned char* smem, int lane) {
  bool ok = j < a.M;
  int h[3] = {0, 0, 0};
  float ar = 0.f;
  AxisNodes<float> s[3];
  if (ok) {
    const int64_t m = a.perm[j];
    const float p[3] = {a.x[m], a.x[a.M + m], a.x[2 * a.M + m]};
    ar = a.area[m];
    ok = isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]) && isfinite(ar);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      h[d] = locate_axis(a.g.ax[d], p[d]);
      ok = ok && support_ok(a.g.ax[d], h[d]);
    }
    if (ok) {
#pragma unroll
      for (int d = 0; d < 3; ++d) s[d] = axis_nodes(a.g.ax[d], h[d], p[d]);
    } else {
      for (int k = 0; k < 27; ++k) a.phi[k * a.cap + j] = 0.f;
      a.c[j] = 0.f;
      a.home[j] = -1;
    }
  }
  float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (ok) {
    // Spacing features of the class axis c and the reference axis u
    // (selected without indexing the node array by a runtime axis).
    const int c = a.ax.c, u = a.ax.u;
    const float wc0 = c == 0 ? s[0].w[0] : (c == 1 ? s[1].w[0] : s[2].w[0]);
    const float wc1 = c == 0 ? s[0].w[1] : (c == 1 ? s[1].w[1] : s[2].w[1]);
    const float wc2 = c == 0 ? s[0].w[2] : (c == 1 ? s[1].w[2] : s[2].w[2]);
    const float wu1 = u == 0 ? s[0].w[1] : (u == 1 ? s[1].w[1] : s[2].w[1]);
    f[0] = s[0].t;
    f[1] = s[1].t;
    f[2] = s[2].t;
    f[3] = logf(wc0 / wc1);
    f[4] = logf(wc2 / wc1);
    f[5] = logf(wc1 / wu1);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) feat[lane * 8 + i] = f[i];
  __syncwarp();
  mlp_warp_bf16(feat, Y, smem);
  __syncwarp();
  if (!ok) return;
  // Projection onto {sum phi = 1, sum phi xi = 0}: G = P^T P factorises per
  // axis (S1_d = sum_a xi_d,a, S2_d = sum_a xi_d,a^2), r = P^T phi - e_0,
  // phi <- phi - P G^-1 r.
  float S1[3], S2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    S1[d] = s[d].xi[0] + s[d].xi[1] + s[d].xi[2];
    S2[d] = s[d].xi[0] * s[d].xi[0] + s[d].xi[1] * s[d].xi[1] + s[d].xi[2] * s[d].xi[2];
  }
  float G[10] = {27.f, 9.f * S1[0], 9.f * S2[0], 9.f * S1[1], 3.f * S1[0] * S1[1], 9.f * S2[1],
                 9.f * S1[2], 3.f * S1[0] * S1[2], 3.f * S1[1] * S1[2], 9.f * S2[2]};
  const float* yr = Y + lane * 33;
  float r[4] = {-1.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int cz = 0; cz < 3; ++cz)
#pragma unroll
    for (int cy = 0; cy < 3; ++cy)
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) {
        const float v = yr[9 * cz + 3 * cy + cx];
        r[0] += v;
        r[1] += v * s[0].xi[cx];
        r[2] += v * s[1].xi[cy];
        r[3] += v * s[2].xi[cz];
      }
  // The gate: the raw network output's linear-reproduction residual (before
  // any projection); a marker above residual_max (or not finite) takes exact-MLS.
  const float rraw = fmaxf(fmaxf(fabsf(r[0]), fabsf(r[1])), fmaxf(fabsf(r[2]), fabsf(r[3])));
  Chol4<float> ch;
  ch.factor(G);
  float lam[4];
  ch.solve(r, lam);
  float res[4] = {-1.f, 0.f, 0.f, 0.f};
  float phi[27];
#pragma unroll
  for (int cz = 0; cz < 3; ++cz)
#pragma unroll
    for (int cy = 0; cy < 3; ++cy)
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) {
        const int k = 9 * cz + 3 * cy + cx;
        const float v = yr[k] - (lam[0] + lam[1] * s[0].xi[cx] + lam[2] * s[1].xi[cy] + lam[3] * s[2].xi[cz]);
        phi[k] = v;
        res[0] += v;
        res[1] += v * s[0].xi[cx];
        res[2] += v * s[1].xi[cy];
        res[3] += v * s[2].xi[cz];
      }
  // After the projection the residual is at rounding level; it is checked only
  // for finiteness (a non-finite projection also takes exact-MLS).
  const float rproj = fmaxf(fmaxf(fabsf(res[0]), fabsf(res[1])), fmaxf(fabsf(res[2]), fabsf(res[3])));
  ScaleSums<float> sums;
  if (!(rraw <= a.residual_max) || !isfinite(rproj)) {
    float w[3][3], y[4];
    const bool good = exact_solve<float>(s, a.inv_eps2, 1, w, y, nullptr);
    if (good)
      exact_emit(s, w, y, [&](int q, int b, int cz, float v) { phi[9 * cz + 3 * b + q] = v; });
    else
      for (int k = 0; k < 27; ++k) phi[k] = 0.f;
    atomicAdd(&a.status[3], 1ULL);
  }
#pragma unroll
  for (int cz = 0; cz < 3; ++cz)
#pragma unroll
    for (int cy = 0; cy < 3; ++cy)
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) {
        const int k = 9 * cz + 3 * cy + cx;
        a.phi[k * a.cap + j] = phi[k];
        sums.add(s, cx, cy, cz, phi[k]);
      }
  a.c[j] = sums.vol != 0.f ? sums.scale(s, ar) : 0.f;
  a.home[j] = (h[2] * a.g.ax[1].n + h[1]) * a.g.ax[0].n + h[0];
}

// Persistent blocks: each copies the packed weights into shared memory once
// and then walks chunks of kMlpThreads markers (one launch of one block per
// chunk would copy the 16 KB of weights again for every 128 markers).
__global__ void __launch_bounds__(kMlpThreads) k_build_surrogate(SurrogateArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_pack(smem, a.pack);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* feat = reinterpret_cast<float*>(smem + kPackBytes) + warp * (kWarpFeat + kWarpY);
  float* Y = feat + kWarpFeat;
  for (int64_t base = (int64_t)blockIdx.x * kMlpThreads; base < a.M; base += (int64_t)gridDim.x * kMlpThreads) {
    __syncwarp();  // the previous chunk's reads of feat and Y are done
    surrogate_marker(a, base + threadIdx.x, feat, Y, smem, lane);
  }
}

static int g_surrogate_grid = 0;  // resident blocks of k_build_surrogate on the device (set by mlp_configure)

// ---- host launchers ----------------------------------------------------------------
static SurrogateAxes surrogate_axes(const mls_ctx* ctx) {
  SurrogateAxes ax;
  ax.c = ctx->class_axis >= 0 ? ctx->class_axis : 2;
  ax.u = ax.c == 0 ? 1 : 0;
  return ax;
}

int surrogate_class_axis(mls_ctx* ctx) {
  int axis = -1, nonuni = 0;
  for (int d = 0; d < 3; ++d)
    if (!ctx->uniform[d]) {
      axis = d;
      ++nonuni;
    }
  if (nonuni > 1) return -2;
  ctx->class_axis = axis;
  return axis;
}

cudaError_t launch_mlp_samples(const mls_ctx* ctx, int64_t first, int64_t count, uint64_t seed, float* X, float* T,
                               cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const SurrogateAxes ax = surrogate_axes(ctx);
  const int n = ctx->n[ax.c];
  const int lo = ctx->periodic[ax.c] ? 0 : 1;
  const int span = ctx->periodic[ax.c] ? n : n - 2;
  const unsigned grid = (unsigned)((count + 127) / 128);
  k_mlp_samples<<<grid, 128, 0, s>>>(device_grid<double>(ctx), ax, lo, span, first, count, seed,
                                     1.0 / (ctx->opt.eps * ctx->opt.eps), X, T);
  return cudaGetLastError();
}

static size_t fwd_smem() { return (size_t)(kParams + 1 + 2 * kH * kMlpThreads + kOut * kMlpThreads) * 4; }

cudaError_t mlp_configure() {
  cudaError_t e;
  const int sm = (int)fwd_smem();
  if ((e = cudaFuncSetAttribute(k_mlp_fwd<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_mlp_fwd<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_mlp_fwd<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_mlp_forward_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, kBf16Smem)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_build_surrogate, cudaFuncAttributeMaxDynamicSharedMemorySize, kBf16Smem)) !=
      cudaSuccess)
    return e;
  int per_sm = 0, sms = 0, dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_surrogate, kMlpThreads, kBf16Smem)) !=
      cudaSuccess)
    return e;
  g_surrogate_grid = (per_sm > 0 ? per_sm : 1) * sms;
  return cudaSuccess;
}

size_t mlp_pack_bytes() { return kPackBytes; }
size_t mlp_train_floats(int B) { return (size_t)B * (kIn + 4 * kH + kOut); }

static TrainBuffers train_buffers(float* base, int B) {
  TrainBuffers tb;
  tb.Xb = base;
  tb.H1 = tb.Xb + (size_t)kIn * B;
  tb.H2 = tb.H1 + (size_t)kH * B;
  tb.dY = tb.H2 + (size_t)kH * B;
  tb.dZ1 = tb.dY + (size_t)kOut * B;
  tb.dZ2 = tb.dZ1 + (size_t)kH * B;
  return tb;
}

// grad = dL/dtheta and *loss_sum += sum of squared residuals for one batch.
cudaError_t launch_mlp_grad(const float* theta, const float* X, const float* T, int64_t n_all, int B, bool gather,
                            uint64_t draw_base, uint64_t seed, float* work, float* grad, float* loss_sum,
                            cudaStream_t s) {
  const TrainBuffers tb = train_buffers(work, B);
  cudaError_t e = cudaMemsetAsync(grad, 0, kParams * sizeof(float), s);
  if (e != cudaSuccess) return e;
  const unsigned nb = (unsigned)((B + kMlpThreads - 1) / kMlpThreads);
  if (gather)
    k_mlp_fwd<true, true><<<nb, kMlpThreads, fwd_smem(), s>>>(theta, X, T, n_all, B, draw_base, seed, tb, nullptr,
                                                              loss_sum);
  else
    k_mlp_fwd<true, false><<<nb, kMlpThreads, fwd_smem(), s>>>(theta, X, T, n_all, B, draw_base, seed, tb, nullptr,
                                                               loss_sum);
  const int chunk = 256;
  dim3 g((kParams + kMlpThreads - 1) / kMlpThreads, (B + chunk - 1) / chunk);
  k_mlp_wgrad<<<g, kMlpThreads, 0, s>>>(B, chunk, tb, grad);
  return cudaGetLastError();
}

__global__ void k_scale1(float* v, float s) { *v *= s; }

cudaError_t launch_scale1(float* v, float s, cudaStream_t st) {
  k_scale1<<<1, 1, 0, st>>>(v, s);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, const float* grad, float* m, float* v, float lr, float bc1, float bc2,
                        cudaStream_t s) {
  k_adam<<<(kParams + 255) / 256, 256, 0, s>>>(theta, grad, m, v, lr, bc1, bc2);
  return cudaGetLastError();
}

cudaError_t launch_mlp_pack(const float* theta, unsigned char* pack, cudaStream_t s) {
  k_mlp_pack<<<1, 256, 0, s>>>(theta, pack);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* theta, const unsigned char* pack, const float* X, int B, int mode,
                               float* Y, cudaStream_t s) {
  const unsigned nb = (unsigned)((B + kMlpThreads - 1) / kMlpThreads);
  if (mode == MLS_F32) {
    TrainBuffers none{};
    k_mlp_fwd<false, false><<<nb, kMlpThreads, fwd_smem(), s>>>(theta, X, nullptr, B, B, 0, 0, none, Y, nullptr);
  } else {
    k_mlp_forward_bf16<<<nb, kMlpThreads, kBf16Smem, s>>>(pack, X, B, Y);
  }
  return cudaGetLastError();
}

cudaError_t launch_build_surrogate(const mls_ctx* ctx, mls_transfer* T, const void* x, const void* area, int64_t M,
                                   cudaStream_t s) {
  SurrogateArgs a;
  a.g = device_grid<float>(ctx);
  a.ax = surrogate_axes(ctx);
  a.x = (const float*)x;
  a.area = (const float*)area;
  a.perm = T->perm;
  a.M = M;
  a.cap = T->cap;
  a.phi = (float*)T->phi;
  a.c = (float*)T->c;
  a.home = T->home;
  a.status = T->status;
  a.inv_eps2 = (float)(1.0 / (ctx->opt.eps * ctx->opt.eps));
  a.residual_max = (float)ctx->opt.residual_max;
  a.pack = ctx->mlp_pack;
  const int64_t chunks = (M + kMlpThreads - 1) / kMlpThreads;
  const int64_t resident = g_surrogate_grid > 0 ? g_surrogate_grid : chunks;
  const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(chunks, resident));
  k_build_surrogate<<<nb, kMlpThreads, kBf16Smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mls
