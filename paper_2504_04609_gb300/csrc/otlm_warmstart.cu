// C ABI of the learned warm start (declared in include/otlm.h): a 4-layer MLP trained on solved
// problems to predict the initial target potential g / eps and log w (kernels in mlp.cuh).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <new>

#include "../../include/otlm.h"
#include "mlp.cuh"

using namespace otlm::mlp;

struct otlm_ws_ctx {
  int n = 0, k = 0, H = 0, batch_max = 0;
  cudaStream_t stream = nullptr;
  int d[LAYERS + 1] = {};
  size_t woff[LAYERS] = {}, boff[LAYERS] = {}, nparams = 0;
  void* mem = nullptr;
  float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
  __nv_bfloat16* P16 = nullptr;
  float* act[LAYERS + 1] = {};
  float* pre[LAYERS] = {};
  float* dh[2] = {};
  float *mean = nullptr, *stdv = nullptr, *part = nullptr, *loss_scale = nullptr;
  long long step = 0;
};

namespace {

constexpr int LOSS_PARTS = 296;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

void forward(otlm_ws_ctx* w, int batch, const float* y) {
  cudaStream_t s = w->stream;
  features_kernel<<<batch, 256, 0, s>>>(y, w->n, w->act[0]);
  for (int l = 0; l < LAYERS; ++l) {
    const int din = w->d[l], dout = w->d[l + 1];
    const bool hidden = l < LAYERS - 1;
    gemm<__nv_bfloat16>(s, batch, dout, din, w->act[l], din, 1, w->P16 + w->woff[l], 1, din, w->act[l + 1], dout,
                        w->P + w->boff[l], hidden ? w->pre[l + 1] : nullptr, hidden);
  }
}

// forward, loss and gradients into w->G; loss (and 2/count) in w->loss_scale
void backward(otlm_ws_ctx* w, int batch, const float* y, const float* target) {
  cudaStream_t s = w->stream;
  forward(w, batch, y);
  const int dz = w->d[LAYERS];
  loss_kernel<<<LOSS_PARTS, 256, 0, s>>>(w->act[LAYERS], target, w->mean, w->stdv, batch, dz, w->dh[0], w->part,
                                         w->part + LOSS_PARTS);
  loss_finish_kernel<<<1, 32, 0, s>>>(w->part, w->part + LOSS_PARTS, LOSS_PARTS, w->loss_scale);
  scale_kernel<<<1184, 256, 0, s>>>(w->dh[0], (size_t)batch * dz, w->loss_scale + 1);
  int cur = 0;
  for (int l = LAYERS - 1; l >= 0; --l) {
    const int din = w->d[l], dout = w->d[l + 1];
    float* dcur = w->dh[cur];
    // dW[o][i] = sum_b dcur[b][o] act[l][b][i]
    gemm<float>(s, dout, din, batch, dcur, 1, dout, w->act[l], din, 1, w->G + w->woff[l], din);
    colsum_rows_kernel<<<(dout + 255) / 256, 256, 0, s>>>(dcur, batch, dout, w->G + w->boff[l]);
    if (l > 0) {
      float* dnext = w->dh[cur ^ 1];
      // dprev[b][i] = sum_o dcur[b][o] W[o][i]  (the BF16 weights the forward pass used)
      gemm<__nv_bfloat16>(s, batch, din, dout, dcur, dout, 1, w->P16 + w->woff[l], din, 1, dnext, din);
      gelu_back_kernel<<<1184, 256, 0, s>>>(dnext, w->pre[l], (size_t)batch * din);
      cur ^= 1;
    }
  }
}

}  // namespace

extern "C" {

int otlm_ws_create(otlm_ws* out, int n, int k, int width, int batch_max, unsigned long long seed, void* stream) {
  if (!out) return OTLM_EINVAL;
  *out = nullptr;
  if (n < 2 || k < 1 || width < 1 || batch_max < 1) return OTLM_EINVAL;
  otlm_ws_ctx* w = new (std::nothrow) otlm_ws_ctx;
  if (!w) return OTLM_ENOMEM;
  w->n = n; w->k = k; w->H = width; w->batch_max = batch_max;
  w->stream = static_cast<cudaStream_t>(stream);
  const int d[LAYERS + 1] = {n + 1, width, width, width, n + k};
  size_t off = 0;
  int dmax = 0;
  for (int l = 0; l <= LAYERS; ++l) {
    w->d[l] = d[l];
    dmax = dmax > d[l] ? dmax : d[l];
  }
  for (int l = 0; l < LAYERS; ++l) {
    w->woff[l] = off;
    off += (size_t)d[l + 1] * d[l];
    w->boff[l] = off;
    off += d[l + 1];
  }
  w->nparams = off;
  size_t bytes = 4 * align256(4 * off) + align256(2 * off);
  size_t actb = 0;
  for (int l = 0; l <= LAYERS; ++l) actb += align256(4 * (size_t)batch_max * d[l]);
  for (int l = 1; l < LAYERS; ++l) actb += align256(4 * (size_t)batch_max * d[l]);
  actb += 2 * align256(4 * (size_t)batch_max * dmax);
  bytes += actb + 2 * align256(4 * (size_t)(n + k)) + align256(4 * 2 * LOSS_PARTS) + 256;
  if (cudaMalloc(&w->mem, bytes) != cudaSuccess) {
    delete w;
    return OTLM_ENOMEM;
  }
  char* p = static_cast<char*>(w->mem);
  auto take = [&](size_t b) { char* r = p; p += align256(b); return r; };
  w->P = (float*)take(4 * off);
  w->G = (float*)take(4 * off);
  w->M = (float*)take(4 * off);
  w->V = (float*)take(4 * off);
  w->P16 = (__nv_bfloat16*)take(2 * off);
  for (int l = 0; l <= LAYERS; ++l) w->act[l] = (float*)take(4 * (size_t)batch_max * d[l]);
  for (int l = 1; l < LAYERS; ++l) w->pre[l] = (float*)take(4 * (size_t)batch_max * d[l]);
  w->dh[0] = (float*)take(4 * (size_t)batch_max * dmax);
  w->dh[1] = (float*)take(4 * (size_t)batch_max * dmax);
  w->mean = (float*)take(4 * (size_t)(n + k));
  w->stdv = (float*)take(4 * (size_t)(n + k));
  w->part = (float*)take(4 * 2 * LOSS_PARTS);
  w->loss_scale = (float*)take(256);
  cudaStream_t s = w->stream;
  cudaError_t e = cudaMemsetAsync(w->P, 0, 4 * off, s);
  for (int l = 0; l < LAYERS && e == cudaSuccess; ++l) {
    const float a = std::sqrt(6.f / (float)(d[l] + d[l + 1]));
    init_kernel<<<1184, 256, 0, s>>>(w->P + w->woff[l], (size_t)d[l + 1] * d[l], a, seed + 0x1000000ull * (l + 1));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(w->M, 0, 4 * off, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->V, 0, 4 * off, s);
  to_bf16_kernel<<<1184, 256, 0, s>>>(w->P, w->P16, off);
  // identity normalisation (mean 0, std 1) until the caller sets one
  if (e == cudaSuccess) e = cudaMemsetAsync(w->mean, 0, 4 * (size_t)(n + k), s);
  if (e == cudaSuccess) {
    fill_kernel<<<(n + k + 255) / 256, 256, 0, s>>>(w->stdv, (size_t)(n + k), 1.f);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaFree(w->mem);
    delete w;
    return OTLM_ECUDA;
  }
  *out = w;
  return OTLM_OK;
}

void otlm_ws_destroy(otlm_ws w) {
  if (!w) return;
  cudaStreamSynchronize(w->stream);
  cudaFree(w->mem);
  delete w;
}

long long otlm_ws_num_params(otlm_ws w) { return w ? (long long)w->nparams : -1; }

int otlm_ws_set_normalization(otlm_ws w, const float* mean, const float* stdv) {
  if (!w || !mean || !stdv) return OTLM_EINVAL;
  const size_t b = 4 * (size_t)(w->n + w->k);
  if (cudaMemcpyAsync(w->mean, mean, b, cudaMemcpyDeviceToDevice, w->stream) != cudaSuccess ||
      cudaMemcpyAsync(w->stdv, stdv, b, cudaMemcpyDeviceToDevice, w->stream) != cudaSuccess)
    return OTLM_ECUDA;
  return OTLM_OK;
}

int otlm_ws_get_params(otlm_ws w, float* out) {
  if (!w || !out) return OTLM_EINVAL;
  return cudaMemcpyAsync(out, w->P, 4 * w->nparams, cudaMemcpyDeviceToDevice, w->stream) == cudaSuccess ? OTLM_OK
                                                                                                          : OTLM_ECUDA;
}

int otlm_ws_set_params(otlm_ws w, const float* in) {
  if (!w || !in) return OTLM_EINVAL;
  if (cudaMemcpyAsync(w->P, in, 4 * w->nparams, cudaMemcpyDeviceToDevice, w->stream) != cudaSuccess)
    return OTLM_ECUDA;
  to_bf16_kernel<<<1184, 256, 0, w->stream>>>(w->P, w->P16, w->nparams);
  return cudaGetLastError() == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}

int otlm_ws_gradients(otlm_ws w, int batch, const float* y, const float* target, float* grad_out, float* loss_out) {
  if (!w || !y || !target || batch < 1 || batch > w->batch_max) return OTLM_EINVAL;
  backward(w, batch, y, target);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && grad_out)
    e = cudaMemcpyAsync(grad_out, w->G, 4 * w->nparams, cudaMemcpyDeviceToDevice, w->stream);
  if (e == cudaSuccess && loss_out) e = cudaMemcpyAsync(loss_out, w->loss_scale, 4, cudaMemcpyDeviceToDevice, w->stream);
  return e == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}

int otlm_ws_train_step(otlm_ws w, int batch, const float* y, const float* target, double lr, double weight_decay,
                       float* loss_out) {
  if (!w || !y || !target || batch < 1 || batch > w->batch_max || !(lr > 0) || !(weight_decay >= 0))
    return OTLM_EINVAL;
  backward(w, batch, y, target);
  w->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - std::pow(b1, (float)w->step), bc2 = 1.f - std::pow(b2, (float)w->step);
  adamw_kernel<<<1184, 256, 0, w->stream>>>(w->P, w->G, w->M, w->V, w->P16, w->nparams, (float)lr, b1, b2, 1e-8f,
                                            (float)weight_decay, bc1, bc2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && loss_out) e = cudaMemcpyAsync(loss_out, w->loss_scale, 4, cudaMemcpyDeviceToDevice, w->stream);
  return e == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}

int otlm_ws_predict(otlm_ws w, int batch, const float* y, double eps, const float* cold_w, float* g0, float* w0) {
  if (!w || !y || !cold_w || !g0 || !w0 || batch < 1 || batch > w->batch_max || !(eps > 0)) return OTLM_EINVAL;
  forward(w, batch, y);
  decode_kernel<<<1184, 256, 0, w->stream>>>(w->act[LAYERS], w->mean, w->stdv, batch, w->n, w->k, (float)eps, cold_w,
                                             g0, w0);
  return cudaGetLastError() == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}

}  // extern "C"
