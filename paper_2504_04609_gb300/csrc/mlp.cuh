// Learned warm start: a 4-layer MLP mapping a target spectrum to initial potentials and weights.
//
//   features  x0 = [ n y / sum(y),  log sum(y) ]                        (n + 1)
//   hidden    h_l = GELU(h_{l-1} W_l^T + b_l),  l = 1..3, width H        (erf form of GELU)
//   output    z = h_3 W_4^T + b_4                                        (n + k)
//   targets   t = [ g / eps (n),  log w (k) ] of solved problems, normalised per output,
//             (t - mean) / std; bins whose target is not finite (g = -inf where y = 0 under the
//             KL datafit) are masked out of the loss.
//   loss      mean over unmasked entries of (z - t_norm)^2
// Weights are stored in BF16 for the forward pass (FP32 accumulation) with FP32 master copies
// updated by AdamW.  Training contractions go through one register-tiled SIMT kernel with strided
// operands (C = A B with A(m,k), B(k,n) given by element strides), which covers the forward pass
// (B = W^T), the input gradient (B = W) and the weight gradient (A = dH^T).  Inference runs the
// forward pass on the tcgen05 GEMM (below).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace otlm {
namespace mlp {

constexpr int LAYERS = 4;

// ---- GEMM: C[m][n] (row stride ldc) = sum_k A(m,k) B(k,n) (+ bias[n]) --------------------------
// A(m,k) = A[m * sam + k * sak] (float), B(k,n) = B[k * sbk + n * sbn] (TB = float or bf16).
// Epilogue: PRE != null stores the pre-activation, C = GELU(pre) when gelu, accumulate into C when
// acc_out.  Tile 64 x 64, k-chunk 16, 256 threads, 4 x 4 outputs per thread.
template <typename TB>
__device__ __forceinline__ float ldB(const TB* p) { return static_cast<float>(*p); }
template <>
__device__ __forceinline__ float ldB<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

template <typename TB>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float* A, long long sam, long long sak,
                                                   const TB* B, long long sbk, long long sbn, float* C, int ldc,
                                                   const float* bias, float* pre, int gelu_on, int acc_out) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += BK) {
    // the contiguous dimension of each operand is the fastest-varying thread index (coalesced)
    for (int e = tid; e < BM * BK; e += 256) {
      const int mm = sak == 1 ? e / BK : e % BM, kk = sak == 1 ? e % BK : e / BM;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? A[m * sam + k * sak] : 0.f;
    }
    for (int e = tid; e < BN * BK; e += 256) {
      const int nn = sbk == 1 ? e / BK : e % BN, kk = sbk == 1 ? e % BK : e / BN;
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < N && k < K) ? ldB<TB>(B + k * sbk + n * sbn) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j] + (bias ? bias[n] : 0.f);
      const size_t idx = (size_t)m * ldc + n;
      if (pre) pre[idx] = v;
      if (gelu_on) v = gelu(v);
      C[idx] = acc_out ? C[idx] + v : v;
    }
  }
}

template <typename TB>
inline void gemm(cudaStream_t s, int M, int N, int K, const float* A, long long sam, long long sak, const TB* B,
                 long long sbk, long long sbn, float* C, int ldc, const float* bias = nullptr, float* pre = nullptr,
                 bool gelu_on = false, bool acc_out = false) {
  const dim3 grid((N + 63) / 64, (M + 63) / 64);
  gemm_kernel<TB><<<grid, 256, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, pre, gelu_on, acc_out);
}

// features: x0[b] = [ n y_b / sum(y_b), log sum(y_b) ]  (one CTA per row)
__global__ void features_kernel(const float* y, int n, float* x0) {
  __shared__ float red[32];
  const int b = blockIdx.x;
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += y[(size_t)b * n + i];
  s = block_sum(s, red);
  const float inv = s > 0.f ? (float)n / s : 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x0[(size_t)b * (n + 1) + i] = y[(size_t)b * n + i] * inv;
  if (threadIdx.x == 0) x0[(size_t)b * (n + 1) + n] = s > 0.f ? logf(s) : 0.f;
}

// loss and output gradient: d = 2 (z - t_norm) / count over unmasked entries; per-CTA partial
// loss sums and counts (deterministic: reduced in a fixed order by loss_finish_kernel).
__global__ void loss_kernel(const float* z, const float* t, const float* mean, const float* std_, int rows, int cols,
                            float* dz, float* part_loss, float* part_cnt) {
  __shared__ float red[32];
  float l = 0.f, c = 0.f;
  const size_t total = (size_t)rows * cols;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % cols);
    const float tv = t[e];
    const bool ok = isfinite(tv);
    const float r = ok ? z[e] - (tv - mean[j]) / std_[j] : 0.f;
    dz[e] = r;  // scaled by 2/count in loss_scale_kernel
    l += r * r;
    c += ok ? 1.f : 0.f;
  }
  l = block_sum(l, red);
  c = block_sum(c, red);
  if (threadIdx.x == 0) {
    part_loss[blockIdx.x] = l;
    part_cnt[blockIdx.x] = c;
  }
}

__global__ void loss_finish_kernel(const float* part_loss, const float* part_cnt, int parts, float* loss_scale) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float l = 0.f, c = 0.f;
    for (int i = 0; i < parts; ++i) {
      l += part_loss[i];
      c += part_cnt[i];
    }
    loss_scale[0] = c > 0.f ? l / c : 0.f;      // loss
    loss_scale[1] = c > 0.f ? 2.f / c : 0.f;    // gradient scale
  }
}

__global__ void scale_kernel(float* v, size_t count, const float* scale) {
  const float s = *scale;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    v[e] *= s;
}

// dH *= GELU'(pre)
__global__ void gelu_back_kernel(float* dh, const float* pre, size_t count) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    dh[e] *= gelu_grad(pre[e]);
}

// db[j] = sum_b dz[b][j]  (one thread per column)
__global__ void colsum_rows_kernel(const float* dz, int rows, int cols, float* db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int b = 0; b < rows; ++b) s += dz[(size_t)b * cols + j];
  db[j] = s;
}

// AdamW on the FP32 master parameters, then the BF16 copy of each weight used by the forward pass.
__global__ void adamw_kernel(float* p, const float* g, float* m, float* v, __nv_bfloat16* p16, size_t count, float lr,
                             float b1, float b2, float eps, float wd, float bc1, float bc2) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const float gr = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gr;
    const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    const float upd = (mm / bc1) / (sqrtf(vv / bc2) + eps);
    const float np = p[e] - lr * (upd + wd * p[e]);
    p[e] = np;
    p16[e] = __float2bfloat16_rn(np);
  }
}

__global__ void fill_kernel(float* p, size_t count, float v) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    p[e] = v;
}

__global__ void to_bf16_kernel(const float* p, __nv_bfloat16* p16, size_t count) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    p16[e] = __float2bfloat16_rn(p[e]);
}

// Deterministic initialisation: uniform(-a, a) from a counter-based hash (splitmix64 of
// seed + index), a = sqrt(6 / (fan_in + fan_out)) for weights; biases 0.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void init_kernel(float* p, size_t count, float a, unsigned long long seed) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const double u = (double)(splitmix64(seed + e) >> 11) * (1.0 / 9007199254740992.0);
    p[e] = (float)((2.0 * u - 1.0) * a);
  }
}

// ---- tensor-core forward pass (inference) ------------------------------------------------------
// Each layer is Z = H W^T on gemm3_kernel<KIND_BF16> with A = W (the BF16 weights; their lo part
// is an all-zero buffer, so the three hi/lo products are W times the activations to ~16 bits) and
// B = the activations as a BF16 hi/lo pair, K-major with a row pitch padded to 8 elements (TMA
// rows are 16-byte multiples).  Z may be split over the reduction (partial-sum planes); the
// activation kernel adds the planes in order, the bias and GELU, and writes the next operand.

// Weights of one layer, [out][in] FP32 -> BF16 with the row pitch inp.
__global__ void pad_bf16_kernel(const float* W, int dout, int din, int inp, __nv_bfloat16* out) {
  const size_t total = (size_t)dout * din;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(e / din), i = (int)(e - (size_t)o * din);
    out[(size_t)o * inp + i] = __float2bfloat16_rn(W[e]);
  }
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  *hi = h;
  *lo = __float2bfloat16_rn(v - __bfloat162float(h));
}

// features as the first operand: [n y / sum(y), log sum(y)] as BF16 hi/lo, row pitch inp.
__global__ void features_split_kernel(const float* y, int n, int inp, __nv_bfloat16* hhi, __nv_bfloat16* hlo) {
  __shared__ float red[32];
  const int b = blockIdx.x;
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += y[(size_t)b * n + i];
  s = block_sum(s, red);
  const float inv = s > 0.f ? (float)n / s : 0.f;
  const size_t row = (size_t)b * inp;
  for (int i = threadIdx.x; i < n; i += blockDim.x) split_bf16(y[(size_t)b * n + i] * inv, hhi + row + i, hlo + row + i);
  if (threadIdx.x == 0) split_bf16(s > 0.f ? logf(s) : 0.f, hhi + row + n, hlo + row + n);
}

// v = sum over the `splits` partial-sum planes of Z [rows][dout] + bias; hidden layers write
// GELU(v) as the next BF16 hi/lo operand (row pitch outp), the last layer writes v to zout.
__global__ void act_split_kernel(const float* Z, int splits, size_t plane, int rows, int dout, const float* bias,
                                 __nv_bfloat16* ohi, __nv_bfloat16* olo, int outp, float* zout) {
  const size_t total = (size_t)rows * dout;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / dout), f = (int)(e - (size_t)b * dout);
    float v = 0.f;
    for (int z = 0; z < splits; ++z) v += Z[z * plane + e];
    v += bias[f];
    if (zout) zout[e] = v;
    else split_bf16(gelu(v), ohi + (size_t)b * outp + f, olo + (size_t)b * outp + f);
  }
}

// predictions -> warm start: g0 = eps * (z * std + mean) for the first n outputs (the potential
// g / eps), w0 = exp(z * std + mean) for the last k (log w); non-finite predictions fall back to
// the cold start (g0 = 0, w0 = cold_w) so that a bad network can only cost iterations, and so does
// every row when *fail is set (a tensor-core GEMM of the forward pass gave up a wait).
__global__ void decode_kernel(const float* z, const float* mean, const float* std_, int rows, int n, int k, float eps,
                              const float* cold_w, float* g0, float* w0, const int* fail) {
  const int cols = n + k;
  const size_t total = (size_t)rows * cols;
  const bool failed = fail && *fail;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / cols), j = (int)(e % cols);
    const float v = failed ? CUDART_NAN_F : z[e] * std_[j] + mean[j];
    if (j < n) {
      g0[(size_t)b * n + j] = isfinite(v) ? eps * v : 0.f;
    } else {
      const float wv = expf(v);
      w0[(size_t)b * k + (j - n)] = (isfinite(wv) && wv > 0.f) ? wv : cold_w[(size_t)b * k + (j - n)];
    }
  }
}


// ---- training data: targets of solved problems and their per-output normalisation ------------

// Target row [g / eps (n), log w (k)] of a solved problem: g / eps is clipped below at g_floor
// (far below any potential that matters: the prediction only seeds the iteration); a
// non-finite g (u1 = 0 where y = 0 under the KL datafit) and w <= 0 give -inf, which the loss
// masks out.
__global__ void make_targets_kernel(const float* g, const float* wts, int rows, int n, int k, float inv_eps,
                                    float g_floor, float* t) {
  const int cols = n + k;
  const size_t total = (size_t)rows * cols;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / cols), j = (int)(e % cols);
    float v;
    if (j < n) {
      const float gv = g[(size_t)b * n + j];
      v = isfinite(gv) ? fmaxf(gv * inv_eps, g_floor) : -CUDART_INF_F;
    } else {
      const float wv = wts[(size_t)b * k + (j - n)];
      v = wv > 0.f ? logf(wv) : -CUDART_INF_F;
    }
    t[e] = v;
  }
}

// Per-output mean and standard deviation over the finite entries of targets [rows][cols], in two
// passes (sum and count, then squared deviations), FP64 partial sums per (row chunk, column) added
// in a fixed order; std is floored at 1e-3.  Thread = column (coalesced across a row), blockIdx.y =
// chunk of rows r = chunk, chunk + NORM_CHUNKS, ...
constexpr int NORM_CHUNKS = 128;
__global__ void norm_partial_kernel(const float* t, int rows, int cols, const float* mean, double* part,
                                    int* cnt) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x, z = blockIdx.y;
  if (c >= cols) return;
  double s = 0.0;
  int m = 0;
  const float mu = mean ? mean[c] : 0.f;
  for (int r = z; r < rows; r += NORM_CHUNKS) {
    const float v = t[(size_t)r * cols + c];
    if (isfinite(v)) {
      const double d = mean ? (double)v - (double)mu : (double)v;
      s += mean ? d * d : d;
      ++m;
    }
  }
  part[(size_t)z * cols + c] = s;
  if (cnt) cnt[(size_t)z * cols + c] = m;
}
// pass 1 (std_out == null): mean = sum / count; pass 2: std = sqrt(sum of squares / count)
__global__ void norm_finish_kernel(const double* part, const int* cnt, int cols, float* mean, float* std_out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0;
  long long m = 0;
  for (int z = 0; z < NORM_CHUNKS; ++z) {
    s += part[(size_t)z * cols + c];
    m += cnt[(size_t)z * cols + c];
  }
  const double q = s / (double)(m > 0 ? m : 1);
  if (!std_out) mean[c] = (float)q;
  else std_out[c] = fmaxf((float)sqrt(q), 1e-3f);
}

}  // namespace mlp
}  // namespace otlm
