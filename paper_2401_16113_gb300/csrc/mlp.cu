// The alpha/m predictor: an MLP 6 -> 64 -> 64 -> 2 (ReLU) mapping problem features to
// (log10 alpha, m), trained on the GPU with the kernels below (FP32) and queried in BF16.
// The paper gives guidance only (alpha = 0.1 or 0.01 suffices, tiny alpha amplifies roundoff
// in steps (a)/(c), Sec. 4); the network learns the alpha and restart length that minimise the
// iteration count of the mixed-precision solver, with alpha = 1e-3 as the fallback.
//
// Parameters (FP32, 4738): W1[64][6], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].
// Loss: mean over samples of 1/2 ||y - target||^2 (both in normalised units).
//   k_mlp_fwd_bwd  one CTA per tile of 128 samples: forward and backward of each sample by one
//                  thread (activations in shared memory), then the tile's gradient sums over its
//                  samples, one parameter per thread; partials per tile.
//   k_mlp_reduce   gradient = fixed-order sum of the tile partials (deterministic).
//   k_mlp_adam     Adam (Kingma & Ba) update.
//   k_mlp_fwd      forward only, FP32 or BF16 weights and activations (FP32 accumulation).
#include <cuda_bf16.h>
#include <math.h>

#include <string>
#include <vector>

#include "aao_internal.cuh"

namespace aao {
namespace {

constexpr int kIn = 6, kH = 64, kOut = 2;
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kOut * kH, kParams = oB3 + kOut;  // 4738
constexpr int kTile = 128;
constexpr int kHS = kH + 1;  // per-sample activation stride in shared memory (odd: no bank conflicts)

// feature / target normalisation (documented in include/aao.h)
const double kFeatMean[kIn] = {0.35, 0.04, 1.125, 8.5, 8.0, 0.0};
const double kFeatScale[kIn] = {0.15, 0.023, 0.5, 1.1, 1.4, 0.1};
const double kYMean[kOut] = {-3.0, 25.0};
const double kYScale[kOut] = {1.5, 12.0};

__global__ void __launch_bounds__(kTile) k_mlp_fwd_bwd(const float* __restrict__ P, const float* __restrict__ X,
                                                       const float* __restrict__ Y, const int* __restrict__ idx,
                                                       int B, float inv_count, float* __restrict__ part,
                                                       float* __restrict__ loss_part) {
  extern __shared__ __align__(16) float sm[];
  float* w = sm;                        // kParams
  float* sx = w + kParams;              // kTile x kIn
  float* h1 = sx + kTile * kIn;         // kTile x kHS
  float* h2 = h1 + kTile * kHS;         // kTile x kHS
  float* d1 = h2 + kTile * kHS;         // kTile x kHS  dL/dz1
  float* d2 = d1 + kTile * kHS;         // kTile x kHS  dL/dz2
  float* dy = d2 + kTile * kHS;         // kTile x kOut
  __shared__ float lred[kTile];
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) w[p] = P[p];
  const int s = threadIdx.x;
  const int gs = blockIdx.x * kTile + s;
  const bool valid = gs < B;
  const int row = valid ? (idx ? idx[gs] : gs) : 0;
  for (int i = 0; i < kIn; ++i) sx[s * kIn + i] = valid ? X[(size_t)row * kIn + i] : 0.f;
  __syncthreads();
  float l = 0.f;
  {
    float* a1 = h1 + s * kHS;
    float* a2 = h2 + s * kHS;
    const float* xs = sx + s * kIn;
    for (int j = 0; j < kH; ++j) {
      float z = w[oB1 + j];
      for (int i = 0; i < kIn; ++i) z = fmaf(w[oW1 + j * kIn + i], xs[i], z);
      a1[j] = fmaxf(z, 0.f);
    }
    for (int k = 0; k < kH; ++k) {
      float z = w[oB2 + k];
      for (int j = 0; j < kH; ++j) z = fmaf(w[oW2 + k * kH + j], a1[j], z);
      a2[k] = fmaxf(z, 0.f);
    }
    float g[kOut];
    for (int o = 0; o < kOut; ++o) {
      float z = w[oB3 + o];
      for (int k = 0; k < kH; ++k) z = fmaf(w[oW3 + o * kH + k], a2[k], z);
      const float e = valid ? z - Y[(size_t)row * kOut + o] : 0.f;
      l = fmaf(0.5f * e, e, l);
      g[o] = e * inv_count;
      dy[s * kOut + o] = g[o];
    }
    float* e2 = d2 + s * kHS;
    for (int k = 0; k < kH; ++k) {
      float v = 0.f;
      for (int o = 0; o < kOut; ++o) v = fmaf(w[oW3 + o * kH + k], g[o], v);
      e2[k] = a2[k] > 0.f ? v : 0.f;
    }
    float* e1 = d1 + s * kHS;
    for (int j = 0; j < kH; ++j) {
      float v = 0.f;
      for (int k = 0; k < kH; ++k) v = fmaf(w[oW2 + k * kH + j], e2[k], v);
      e1[j] = a1[j] > 0.f ? v : 0.f;
    }
  }
  lred[s] = l;
  __syncthreads();
  // the tile's gradient: one parameter per thread, summed over the tile's samples in order
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) {
    float acc = 0.f;
    if (p < oB1) {
      const int j = (p - oW1) / kIn, i = (p - oW1) % kIn;
      for (int t = 0; t < kTile; ++t) acc = fmaf(d1[t * kHS + j], sx[t * kIn + i], acc);
    } else if (p < oW2) {
      const int j = p - oB1;
      for (int t = 0; t < kTile; ++t) acc += d1[t * kHS + j];
    } else if (p < oB2) {
      const int k = (p - oW2) / kH, j = (p - oW2) % kH;
      for (int t = 0; t < kTile; ++t) acc = fmaf(d2[t * kHS + k], h1[t * kHS + j], acc);
    } else if (p < oW3) {
      const int k = p - oB2;
      for (int t = 0; t < kTile; ++t) acc += d2[t * kHS + k];
    } else if (p < oB3) {
      const int o = (p - oW3) / kH, k = (p - oW3) % kH;
      for (int t = 0; t < kTile; ++t) acc = fmaf(dy[t * kOut + o], h2[t * kHS + k], acc);
    } else {
      const int o = p - oB3;
      for (int t = 0; t < kTile; ++t) acc += dy[t * kOut + o];
    }
    part[(size_t)blockIdx.x * kParams + p] = acc;
  }
  if (threadIdx.x == 0) {
    float a = 0.f;
    for (int t = 0; t < kTile; ++t) a += lred[t];
    loss_part[blockIdx.x] = a;
  }
}

__global__ void k_mlp_reduce(const float* __restrict__ part, const float* __restrict__ loss_part, int tiles,
                             float inv_count, float* __restrict__ grad, float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kParams) {
    float a = 0.f;
    for (int t = 0; t < tiles; ++t) a += part[(size_t)t * kParams + p];
    grad[p] = a;
  }
  if (p == 0) {
    float a = 0.f;
    for (int t = 0; t < tiles; ++t) a += loss_part[t];
    *loss = a * inv_count;
  }
}

__global__ void k_mlp_adam(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m1,
                           float* __restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  const float gp = g[p];
  const float a = b1 * m1[p] + (1.f - b1) * gp;
  const float v = b2 * m2[p] + (1.f - b2) * gp * gp;
  m1[p] = a;
  m2[p] = v;
  P[p] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

template <bool BF16>
__device__ __forceinline__ float q(float v) {
  return BF16 ? __bfloat162float(__float2bfloat16(v)) : v;
}

// forward; with BF16 the weights and every activation are rounded to bfloat16 (accumulation FP32)
template <bool BF16>
__global__ void __launch_bounds__(128) k_mlp_fwd(const float* __restrict__ P, const float* __restrict__ X, int B,
                                                 float* __restrict__ Y) {
  __shared__ float w[kParams];
  for (int p = threadIdx.x; p < kParams; p += blockDim.x) w[p] = q<BF16>(P[p]);
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  float x[kIn], a1[kH];
  for (int i = 0; i < kIn; ++i) x[i] = q<BF16>(X[(size_t)s * kIn + i]);
  for (int j = 0; j < kH; ++j) {
    float z = w[oB1 + j];
    for (int i = 0; i < kIn; ++i) z = fmaf(w[oW1 + j * kIn + i], x[i], z);
    a1[j] = q<BF16>(fmaxf(z, 0.f));
  }
  float y0 = w[oB3], y1 = w[oB3 + 1];
  for (int k = 0; k < kH; ++k) {
    float z = w[oB2 + k];
    for (int j = 0; j < kH; ++j) z = fmaf(w[oW2 + k * kH + j], a1[j], z);
    const float a2 = q<BF16>(fmaxf(z, 0.f));
    y0 = fmaf(w[oW3 + k], a2, y0);
    y1 = fmaf(w[oW3 + kH + k], a2, y1);
  }
  Y[(size_t)s * kOut] = y0;
  Y[(size_t)s * kOut + 1] = y1;
}

}  // namespace

struct Mlp {
  float *P = nullptr, *m1 = nullptr, *m2 = nullptr, *g = nullptr, *part = nullptr, *lpart = nullptr, *loss = nullptr;
  float *xq = nullptr, *yq = nullptr;
  int* idx = nullptr;
  int part_tiles = 0, idx_cap = 0;
  long step = 0;
  cudaStream_t s = 0;
};

}  // namespace aao

struct aao_mlp {
  aao::Mlp M;
};

using namespace aao;

namespace {

size_t fb_smem() { return sizeof(float) * (kParams + kTile * kIn + 4 * kTile * kHS + kTile * kOut); }

int ensure_part(Mlp& M, int tiles) {
  if (M.part_tiles >= tiles) return AAO_OK;
  if (M.part) cudaFree(M.part);
  if (M.lpart) cudaFree(M.lpart);
  M.part = M.lpart = nullptr;
  M.part_tiles = 0;
  AAO_TRY_CUDA(cudaMalloc(&M.part, sizeof(float) * (size_t)tiles * kParams));
  AAO_TRY_CUDA(cudaMalloc(&M.lpart, sizeof(float) * tiles));
  M.part_tiles = tiles;
  return AAO_OK;
}

// gradient of the loss over samples idx[0..B) (or 0..B) into M.g, loss into M.loss
int grad_pass(Mlp& M, const float* X, const float* Y, const int* idx, int B) {
  const int tiles = (B + kTile - 1) / kTile;
  AAO_TRY(ensure_part(M, tiles));
  const size_t smem = fb_smem();
  AAO_TRY_CUDA(cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_mlp_fwd_bwd<<<tiles, kTile, smem, M.s>>>(M.P, X, Y, idx, B, 1.f / B, M.part, M.lpart);
  AAO_CHECK_LAUNCH();
  k_mlp_reduce<<<(kParams + 255) / 256, 256, 0, M.s>>>(M.part, M.lpart, tiles, 1.f / B, M.g, M.loss);
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

// 64-bit LCG with a Fisher-Yates shuffle: the minibatch order of each epoch
void shuffle(std::vector<int>& v, unsigned long long& st) {
  for (int i = (int)v.size() - 1; i > 0; --i) {
    st = st * 6364136223846793005ULL + 1442695040888963407ULL;
    const int j = (int)((st >> 33) % (unsigned long long)(i + 1));
    std::swap(v[i], v[j]);
  }
}

}  // namespace

extern "C" {

int aao_mlp_create(const float* init, void* stream, aao_mlp** out) {
  if (!out || !init) { set_error("aao_mlp_create: null argument"); return AAO_EINVAL; }
  *out = nullptr;
  aao_mlp* h = new aao_mlp();
  Mlp& M = h->M;
  M.s = (cudaStream_t)stream;
  auto fail = [&](int code) {
    float* bufs[] = {M.P, M.m1, M.m2, M.g, M.loss};
    for (float* b : bufs) if (b) cudaFree(b);
    delete h;
    return code;
  };
  if (cudaMalloc(&M.P, sizeof(float) * kParams) != cudaSuccess || cudaMalloc(&M.m1, sizeof(float) * kParams) != cudaSuccess ||
      cudaMalloc(&M.m2, sizeof(float) * kParams) != cudaSuccess || cudaMalloc(&M.g, sizeof(float) * kParams) != cudaSuccess ||
      cudaMalloc(&M.loss, sizeof(float)) != cudaSuccess) {
    set_error("aao_mlp_create: device allocation failed");
    return fail(AAO_ENOMEM);
  }
  if (cudaMemcpyAsync(M.P, init, sizeof(float) * kParams, cudaMemcpyHostToDevice, M.s) != cudaSuccess ||
      cudaMemsetAsync(M.m1, 0, sizeof(float) * kParams, M.s) != cudaSuccess ||
      cudaMemsetAsync(M.m2, 0, sizeof(float) * kParams, M.s) != cudaSuccess ||
      cudaStreamSynchronize(M.s) != cudaSuccess) {
    set_error("aao_mlp_create: upload failed");
    return fail(AAO_ECUDA);
  }
  *out = h;
  return AAO_OK;
}

int aao_mlp_destroy(aao_mlp* h) {
  if (!h) return AAO_OK;
  Mlp& M = h->M;
  cudaStreamSynchronize(M.s);
  float* bufs[] = {M.P, M.m1, M.m2, M.g, M.part, M.lpart, M.loss, M.xq, M.yq};
  for (float* b : bufs) if (b) cudaFree(b);
  if (M.idx) cudaFree(M.idx);
  delete h;
  return AAO_OK;
}

int aao_mlp_params(aao_mlp* h, float* host_out) {
  if (!h || !host_out) { set_error("aao_mlp_params: null argument"); return AAO_EINVAL; }
  AAO_TRY_CUDA(cudaMemcpyAsync(host_out, h->M.P, sizeof(float) * kParams, cudaMemcpyDeviceToHost, h->M.s));
  AAO_TRY_CUDA(cudaStreamSynchronize(h->M.s));
  return AAO_OK;
}

int aao_mlp_grad(aao_mlp* h, const float* X, const float* Y, int B, float* grad_host, float* loss_host) {
  if (!h || !X || !Y || B < 1 || !grad_host || !loss_host) { set_error("aao_mlp_grad: bad argument"); return AAO_EINVAL; }
  AAO_TRY(grad_pass(h->M, X, Y, nullptr, B));
  AAO_TRY_CUDA(cudaMemcpyAsync(grad_host, h->M.g, sizeof(float) * kParams, cudaMemcpyDeviceToHost, h->M.s));
  AAO_TRY_CUDA(cudaMemcpyAsync(loss_host, h->M.loss, sizeof(float), cudaMemcpyDeviceToHost, h->M.s));
  AAO_TRY_CUDA(cudaStreamSynchronize(h->M.s));
  return AAO_OK;
}

int aao_mlp_adam_step(aao_mlp* h, const float* grad_dev, float lr) {
  if (!h || !grad_dev) { set_error("aao_mlp_adam_step: null argument"); return AAO_EINVAL; }
  Mlp& M = h->M;
  ++M.step;
  const float b1 = 0.9f, b2 = 0.999f;
  k_mlp_adam<<<(kParams + 255) / 256, 256, 0, M.s>>>(M.P, grad_dev, M.m1, M.m2, lr, b1, b2, 1e-8f,
                                                      1.f - powf(b1, (float)M.step), 1.f - powf(b2, (float)M.step));
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

int aao_mlp_train(aao_mlp* h, const float* X, const float* Y, int B, int epochs, int minibatch, float lr,
                  unsigned long long seed, float* loss_host) {
  if (!h || !X || !Y || B < 1 || epochs < 1 || minibatch < 1) { set_error("aao_mlp_train: bad argument"); return AAO_EINVAL; }
  Mlp& M = h->M;
  if (M.idx_cap < B) {
    if (M.idx) cudaFree(M.idx);
    M.idx = nullptr;
    AAO_TRY_CUDA(cudaMalloc(&M.idx, sizeof(int) * B));
    M.idx_cap = B;
  }
  std::vector<int> order(B);
  for (int i = 0; i < B; ++i) order[i] = i;
  unsigned long long st = seed;
  int* pinned = nullptr;
  AAO_TRY_CUDA(cudaMallocHost(&pinned, sizeof(int) * B));
  int rc = AAO_OK;
  for (int e = 0; e < epochs && rc == AAO_OK; ++e) {
    shuffle(order, st);
    cudaStreamSynchronize(M.s);  // the pinned order buffer is reused
    memcpy(pinned, order.data(), sizeof(int) * B);
    if (cudaMemcpyAsync(M.idx, pinned, sizeof(int) * B, cudaMemcpyHostToDevice, M.s) != cudaSuccess) { rc = AAO_ECUDA; break; }
    for (int b0 = 0; b0 < B && rc == AAO_OK; b0 += minibatch) {
      const int nb = B - b0 < minibatch ? B - b0 : minibatch;
      rc = grad_pass(M, X, Y, M.idx + b0, nb);
      if (rc == AAO_OK) rc = aao_mlp_adam_step(h, M.g, lr);
    }
  }
  if (rc == AAO_OK) rc = grad_pass(M, X, Y, nullptr, B);
  if (rc == AAO_OK && loss_host) {
    if (cudaMemcpyAsync(loss_host, M.loss, sizeof(float), cudaMemcpyDeviceToHost, M.s) != cudaSuccess) rc = AAO_ECUDA;
  }
  cudaStreamSynchronize(M.s);
  cudaFreeHost(pinned);
  return rc;
}

int aao_mlp_forward(aao_mlp* h, const float* X, float* Y, int B, int bf16) {
  if (!h || !X || !Y || B < 1) { set_error("aao_mlp_forward: bad argument"); return AAO_EINVAL; }
  Mlp& M = h->M;
  if (bf16)
    k_mlp_fwd<true><<<(B + 127) / 128, 128, 0, M.s>>>(M.P, X, B, Y);
  else
    k_mlp_fwd<false><<<(B + 127) / 128, 128, 0, M.s>>>(M.P, X, B, Y);
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

int aao_mlp_normalization(double* feat_mean, double* feat_scale, double* y_mean, double* y_scale) {
  if (!feat_mean || !feat_scale || !y_mean || !y_scale) { set_error("aao_mlp_normalization: null argument"); return AAO_EINVAL; }
  for (int i = 0; i < kIn; ++i) { feat_mean[i] = kFeatMean[i]; feat_scale[i] = kFeatScale[i]; }
  for (int o = 0; o < kOut; ++o) { y_mean[o] = kYMean[o]; y_scale[o] = kYScale[o]; }
  return AAO_OK;
}

int alpha_mlp_predict(aao_mlp* h, const float feats[6], double* alpha, int* m) {
  if (!h || !feats || !alpha || !m) { set_error("alpha_mlp_predict: null argument"); return AAO_EINVAL; }
  Mlp& M = h->M;
  if (!M.xq) {
    AAO_TRY_CUDA(cudaMalloc(&M.xq, sizeof(float) * kIn));
    AAO_TRY_CUDA(cudaMalloc(&M.yq, sizeof(float) * kOut));
  }
  float xn[kIn], y[kOut];
  for (int i = 0; i < kIn; ++i) {
    double v = feats[i];
    if (i == 3 || i == 4) v = log2(v > 1 ? v : 1.0);
    xn[i] = (float)((v - kFeatMean[i]) / kFeatScale[i]);
  }
  AAO_TRY_CUDA(cudaMemcpyAsync(M.xq, xn, sizeof xn, cudaMemcpyHostToDevice, M.s));
  k_mlp_fwd<true><<<1, 128, 0, M.s>>>(M.P, M.xq, 1, M.yq);
  AAO_CHECK_LAUNCH();
  AAO_TRY_CUDA(cudaMemcpyAsync(y, M.yq, sizeof y, cudaMemcpyDeviceToHost, M.s));
  AAO_TRY_CUDA(cudaStreamSynchronize(M.s));
  const double la = y[0] * kYScale[0] + kYMean[0];
  const double mm = y[1] * kYScale[1] + kYMean[1];
  double a = pow(10.0, la);
  if (!(a == a)) a = 1e-3;  // NaN -> the default
  *alpha = a < 1e-5 ? 1e-5 : (a > 0.1 ? 0.1 : a);
  // round up to the next restart choice {5, 10, 20, 30, 40}
  static const int kM[5] = {5, 10, 20, 30, 40};
  int mi = 40;
  for (int c = 0; c < 5; ++c)
    if (mm <= kM[c] + 0.5) { mi = kM[c]; break; }
  *m = mi;
  return AAO_OK;
}

}  // extern "C"
