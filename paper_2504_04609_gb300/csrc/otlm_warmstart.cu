// C ABI of the learned warm start (declared in include/otlm.h): a 4-layer MLP trained on solved
// problems to predict the initial target potential g / eps and log w (kernels in mlp.cuh).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <new>

#include "../../include/otlm.h"
#include "mlp.cuh"
#include "tc_gemm.cuh"

using namespace otlm::mlp;

constexpr int TC_MAX_SPLITS = 16;

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
  // tensor-core forward pass (inference): padded BF16 weights, a zero lo part, activations as BF16
  // hi/lo pairs (ping-pong), split partial sums, and the GEMMs' error flag
  int inp[LAYERS] = {};            // row pitch of layer l's input operand (d[l] rounded up to 8)
  int dmax = 0;                    // widest layer output
  __nv_bfloat16* W16p[LAYERS] = {};
  __nv_bfloat16* zero16 = nullptr;
  __nv_bfloat16 *Hhi[2] = {}, *Hlo[2] = {};
  float* Zs = nullptr;             // [TC_MAX_SPLITS][batch_max][dmax]
  int* tc_err = nullptr;
  bool tc_dirty = true;
  // per-output normalisation statistics: FP64 partial sums and counts per (row chunk, output)
  double* norm_part = nullptr;
  int* norm_cnt = nullptr;            // W16p is stale (weights changed since the last refresh)
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

// Forward pass on the tensor cores into w->act[LAYERS] (inference only: no pre-activations).
cudaError_t forward_tc(otlm_ws_ctx* w, int batch, const float* y) {
  cudaStream_t s = w->stream;
  if (w->tc_dirty) {
    for (int l = 0; l < LAYERS; ++l)
      pad_bf16_kernel<<<1184, 256, 0, s>>>(w->P + w->woff[l], w->d[l + 1], w->d[l], w->inp[l], w->W16p[l]);
    w->tc_dirty = false;
  }
  cudaError_t e = cudaMemsetAsync(w->tc_err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  features_split_kernel<<<batch, 256, 0, s>>>(y, w->n, w->inp[0], w->Hhi[0], w->Hlo[0]);
  const size_t plane = (size_t)w->batch_max * w->dmax;
  int cur = 0;
  for (int l = 0; l < LAYERS; ++l) {
    const int din = w->d[l], dout = w->d[l + 1];
    otlm::tc::GemmArgs g{};
    g.out = w->Zs; g.M = dout; g.N = batch; g.Kd = din; g.ld_out = dout; g.err = w->tc_err;
    g.splits = otlm::tc::choose_splits(((dout + otlm::tc::BM - 1) / otlm::tc::BM) * ((batch + otlm::tc::BN - 1) / otlm::tc::BN),
                                       (din + 63) / 64);
    if (g.splits > TC_MAX_SPLITS) g.splits = TC_MAX_SPLITS;
    g.split_stride = plane;
    e = otlm::tc::launch_gemm3<otlm::tc::KIND_BF16>(w->W16p[l], w->zero16, w->inp[l], w->Hhi[cur], w->Hlo[cur],
                                                    w->inp[l], dout, batch, din, g, s);
    if (e != cudaSuccess) return e;
    const bool last = l == LAYERS - 1;
    act_split_kernel<<<1184, 256, 0, s>>>(w->Zs, g.splits, plane, batch, dout, w->P + w->boff[l],
                                          last ? nullptr : w->Hhi[cur ^ 1], last ? nullptr : w->Hlo[cur ^ 1],
                                          last ? 0 : w->inp[l + 1], last ? w->act[LAYERS] : nullptr);
    cur ^= 1;
  }
  return cudaGetLastError();
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
  size_t w16b = 0, zero_elems = 0;
  int maxp = 0;
  for (int l = 0; l < LAYERS; ++l) {
    w->inp[l] = (d[l] + 7) / 8 * 8;
    w16b += align256(2 * (size_t)d[l + 1] * w->inp[l]);
    const size_t el = (size_t)d[l + 1] * w->inp[l];
    zero_elems = zero_elems > el ? zero_elems : el;
    maxp = maxp > w->inp[l] ? maxp : w->inp[l];
    w->dmax = w->dmax > d[l + 1] ? w->dmax : d[l + 1];
  }
  bytes += w16b + align256(2 * zero_elems) + 4 * align256(2 * (size_t)batch_max * maxp) +
           align256(4 * (size_t)TC_MAX_SPLITS * batch_max * w->dmax) + 256;
  bytes += align256(8 * (size_t)NORM_CHUNKS * (n + k)) + align256(4 * (size_t)NORM_CHUNKS * (n + k));
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
  for (int l = 0; l < LAYERS; ++l) w->W16p[l] = (__nv_bfloat16*)take(2 * (size_t)d[l + 1] * w->inp[l]);
  w->zero16 = (__nv_bfloat16*)take(2 * zero_elems);
  for (int c = 0; c < 2; ++c) {
    w->Hhi[c] = (__nv_bfloat16*)take(2 * (size_t)batch_max * maxp);
    w->Hlo[c] = (__nv_bfloat16*)take(2 * (size_t)batch_max * maxp);
  }
  w->Zs = (float*)take(4 * (size_t)TC_MAX_SPLITS * batch_max * w->dmax);
  w->tc_err = (int*)take(256);
  w->norm_part = (double*)take(8 * (size_t)NORM_CHUNKS * (n + k));
  w->norm_cnt = (int*)take(4 * (size_t)NORM_CHUNKS * (n + k));
  cudaStream_t s = w->stream;
  // the zero lo part of the weights, and zero padding columns of the weights and activations
  // (never read past the tensor maps' extents, cleared all the same)
  cudaError_t e = cudaMemsetAsync(w->W16p[0], 0, w16b + align256(2 * zero_elems) + 4 * align256(2 * (size_t)batch_max * maxp), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->P, 0, 4 * off, s);
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
  w->tc_dirty = true;
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
  w->tc_dirty = true;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && loss_out) e = cudaMemcpyAsync(loss_out, w->loss_scale, 4, cudaMemcpyDeviceToDevice, w->stream);
  return e == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}

int otlm_ws_predict(otlm_ws w, int batch, const float* y, double eps, const float* cold_w, float* g0, float* w0) {
  if (!w || !y || !cold_w || !g0 || !w0 || batch < 1 || batch > w->batch_max || !(eps > 0)) return OTLM_EINVAL;
  if (forward_tc(w, batch, y) != cudaSuccess) return OTLM_ECUDA;
  decode_kernel<<<1184, 256, 0, w->stream>>>(w->act[LAYERS], w->mean, w->stdv, batch, w->n, w->k, (float)eps, cold_w,
                                             g0, w0, w->tc_err);
  return cudaGetLastError() == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}

int otlm_ws_make_targets(otlm_ws w, int batch, const float* g, const float* wts, double eps, double g_floor,
                         float* targets) {
  if (!w || !g || !wts || !targets || batch < 1 || !(eps > 0) || !std::isfinite(eps) || !(g_floor == g_floor))
    return OTLM_EINVAL;
  make_targets_kernel<<<1184, 256, 0, w->stream>>>(g, wts, batch, w->n, w->k, (float)(1.0 / eps), (float)g_floor,
                                                   targets);
  return cudaGetLastError() == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}

int otlm_ws_fit_normalization(otlm_ws w, int rows, const float* targets, float* mean_out, float* std_out) {
  if (!w || !targets || rows < 1) return OTLM_EINVAL;
  const int cols = w->n + w->k;
  const dim3 grid((cols + 255) / 256, NORM_CHUNKS);
  cudaStream_t s = w->stream;
  norm_partial_kernel<<<grid, 256, 0, s>>>(targets, rows, cols, nullptr, w->norm_part, w->norm_cnt);
  norm_finish_kernel<<<(cols + 255) / 256, 256, 0, s>>>(w->norm_part, w->norm_cnt, cols, w->mean, nullptr);
  norm_partial_kernel<<<grid, 256, 0, s>>>(targets, rows, cols, w->mean, w->norm_part, nullptr);
  norm_finish_kernel<<<(cols + 255) / 256, 256, 0, s>>>(w->norm_part, w->norm_cnt, cols, w->mean, w->stdv);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && mean_out)
    e = cudaMemcpyAsync(mean_out, w->mean, 4 * (size_t)cols, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && std_out) e = cudaMemcpyAsync(std_out, w->stdv, 4 * (size_t)cols, cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}

}  // extern "C"
