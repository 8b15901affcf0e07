// Batched scaling iteration with the two kernel applies on the tensor cores (BF16 hi/lo operands,
// FP32 accumulation), for a batch sharing one grid and one dictionary.
//
// Linear domain with a per-problem shift: the source apply is
//   a_pi = sum_j K_ij u1_pj = 2^{M_p} sum_j K_ij V_pj,   V_pj = 2^{G2_pj - M_p},  M_p = max_j G2_pj,
// so every V lies in (0, 1] and the GEMM K V^T (tc_gemm.cuh) returns the raw sums; log2 a_pi =
// M_p + log2(sum).  The target apply is the same with U_pi = 2^{F2_pi - M'_p}.  K is symmetric for
// the squared distance on a grid, so one matrix serves both applies.  Per iteration:
//   prep_src : datafit step from the previous target sums (Table 1), then the source operand V
//   gemm     : source sums into ACC_src[it & 1]
//   mm_tc    : violation from the ratio of raw sums, MM step (Table 2), source step, operand U
//   compact  : drop finished problems
//   gemm     : target sums into ACC_tgt
// A sum that underflows to 0 (possible only when a row's significant terms lie more than ~2^-126
// below the problem's largest term) makes the problem report OTLM_NONFINITE.
#pragma once

#include <cuda_bf16.h>

#include "kernels.cuh"
#include "solver.cuh"
#include "tc_gemm.cuh"

namespace otlm {

struct TcWorkspace {
  __nv_bfloat16 *Khi, *Klo;  // [n][ld]
  __nv_bfloat16 *Vhi, *Vlo;  // [batch][ld], rows in active-slot order (source and target operands)
  float* ACC_src[2];         // [batch][n] raw source sums, ping-pong by iteration parity
  float* ACC_tgt;            // [batch][n] raw target sums
  float* Msrc[2];            // [batch] source shifts, ping-pong
  float* Mtgt;               // [batch] target shifts
  int* err;                  // GEMM error flag
  int ld;                    // row pitch of the BF16 operands (multiple of 64)
};

inline int tc_ld(int n) { return (n + 63) / 64 * 64; }

inline size_t carve_tc_workspace(void* base, int n_max, int batch_max, TcWorkspace* ws) {
  const int ld = tc_ld(n_max);
  size_t off = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* p = b ? b + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  TcWorkspace w;
  w.ld = ld;
  w.Khi = (__nv_bfloat16*)take(2 * (size_t)n_max * ld);
  w.Klo = (__nv_bfloat16*)take(2 * (size_t)n_max * ld);
  w.Vhi = (__nv_bfloat16*)take(2 * (size_t)batch_max * ld);
  w.Vlo = (__nv_bfloat16*)take(2 * (size_t)batch_max * ld);
  w.ACC_src[0] = (float*)take(4 * (size_t)batch_max * n_max);
  w.ACC_src[1] = (float*)take(4 * (size_t)batch_max * n_max);
  w.ACC_tgt = (float*)take(4 * (size_t)batch_max * n_max);
  w.Msrc[0] = (float*)take(4 * (size_t)batch_max);
  w.Msrc[1] = (float*)take(4 * (size_t)batch_max);
  w.Mtgt = (float*)take(4 * (size_t)batch_max);
  w.err = (int*)take(64);
  if (ws) *ws = w;
  return off;
}

// K = 2^{-(xt_i - xt_j)^2} as a BF16 hi/lo pair, [n][ld] (columns >= n left untouched: the
// tensor maps stop at column n).
__global__ void kbuild_kernel(const float* xt, int n, int ld, __nv_bfloat16* Khi, __nv_bfloat16* Klo) {
  const size_t nn = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (size_t)i * n);
    const float d = xt[i] - xt[j];
    const float k = Prec<float>::exp2(-d * d);
    const __nv_bfloat16 hi = __float2bfloat16_rn(k);
    Khi[(size_t)i * ld + j] = hi;
    Klo[(size_t)i * ld + j] = __float2bfloat16_rn(k - __bfloat162float(hi));
  }
}

// max over a block of 256 threads
__device__ __forceinline__ float block_max_f(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : -CUDART_INF_F;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (threadIdx.x == 0) red[0] = v;
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

// Write row `slot` of the operand: 2^{L_j - M} as BF16 hi + lo, where M = max_j L_j.  Returns M.
__device__ __forceinline__ float write_operand(const float* L, int n, int ld, int slot, __nv_bfloat16* Vhi,
                                               __nv_bfloat16* Vlo, float* red) {
  float m = -CUDART_INF_F;
  for (int j = threadIdx.x; j < n; j += blockDim.x) m = fmaxf(m, L[j]);
  m = block_max_f(m, red);
  if (!(m > -CUDART_INF_F)) m = 0.f;  // every term vanishes
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const float v = Prec<float>::exp2(L[j] - m);
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    Vhi[(size_t)slot * ld + j] = hi;
    Vlo[(size_t)slot * ld + j] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
  return m;
}

struct TcIterArgs {
  const int* active;
  const int* n_active;
  int n, k, ld, it, max_iter, datafit, penalty;
  float tol, eps, alpha, kl_coef, tv_bound, lam_over_eps, log_lam_over_eps;
  const float* y;
  const float* D;
  const float* Dt;
  const float* xcol;
  float* G2;
  float* S;
  float* F2;
  float* W;
  float* mass;
  float* err;
  int* done;
  int* iters;
  int* status;
  TcWorkspace t;
};

// Datafit step from the previous target sums (it > 0), then the source operand.
__global__ void __launch_bounds__(256) tc_prep_src_kernel(TcIterArgs A) {
  using P = Prec<float>;
  __shared__ float red[32];
  const int slot = blockIdx.x;
  if (slot >= *A.n_active) return;
  const int p = A.active[slot], n = A.n;
  float* G2 = A.G2 + (size_t)p * n;
  if (A.it > 0) {
    const float* acc = A.t.ACC_tgt + (size_t)p * n;
    const float* y = A.y + (size_t)p * n;
    const float mt = A.t.Mtgt[p];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const float s = acc[j];
      const float v = s > 0.f ? mt + P::log2(s) : P::ninf();
      const float yv = y[j];
      float gn;
      switch (A.datafit) {
        case DF_BALANCED: gn = P::log2(yv) - v; break;
        case DF_KL: gn = A.kl_coef * (P::log2(yv) - v); break;
        case DF_TV: gn = fminf(fmaxf(P::log2(yv) - v, -A.tv_bound), A.tv_bound); break;
        default: {
          const float z = A.log_lam_over_eps + v * float(kLn2) + A.lam_over_eps * yv;
          gn = (A.lam_over_eps * yv - wright_omega<float>(z)) * float(kLog2e);
        }
      }
      G2[j] = gn;
    }
    __syncthreads();
  }
  const float m = write_operand(G2, n, A.t.ld, slot, A.t.Vhi, A.t.Vlo, red);
  if (threadIdx.x == 0) A.t.Msrc[A.it & 1][p] = m;
}

// Violation of the previous iteration's plan and the stopping decision (one CTA per active slot):
// e = sum_i S_i |a_new_i / a_old_i - 1| / sum_i S_i from the raw sums.  The shift difference of
// two nearby FP32 numbers is exact, so the ratio keeps FP32 relative precision.
__global__ void __launch_bounds__(256) tc_violation_kernel(TcIterArgs A) {
  using P = Prec<float>;
  __shared__ float red[32];
  const int slot = blockIdx.x;
  if (slot >= *A.n_active) return;
  const int p = A.active[slot], n = A.n, cur = A.it & 1;
  const float* acc = A.t.ACC_src[cur] + (size_t)p * n;
  const float* acc_old = A.t.ACC_src[cur ^ 1] + (size_t)p * n;
  const float* S = A.S + (size_t)p * n;
  const float f = P::exp2(A.t.Msrc[cur][p] - A.t.Msrc[cur ^ 1][p]);
  float part = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float s = S[i];
    if (s > 0.f) part += s * fabsf(acc[i] / acc_old[i] * f - 1.f);
  }
  part = block_sum(part, red);
  if (threadIdx.x == 0) {
    const float e = part / A.mass[p];
    A.err[p] = e;
    int st = -1;
    if (e != e) st = ST_NONFINITE;
    else if (A.tol > 0.f && e <= A.tol) st = ST_CONVERGED;
    else if (A.it >= A.max_iter) st = ST_MAX_ITER;
    if (st >= 0) {
      A.status[p] = st;
      A.iters[p] = A.it;
      A.done[p] = 1;
    }
  }
}

// MM step, source step and the target operand (one CTA of 256 threads per active slot, after the
// finished problems have been compacted away so that the operand rows match the GEMM's columns).
template <int KQ>
__global__ void __launch_bounds__(256) tc_mm_kernel(TcIterArgs A) {
  using P = Prec<float>;
  constexpr int KP = KQ * 32;
  __shared__ float red_s[8][KP];
  __shared__ float w_s[KP];
  __shared__ float red[32];
  const int slot = blockIdx.x;
  if (slot >= *A.n_active) return;
  const int p = A.active[slot];
  const int n = A.n, k = A.k;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cur = A.it & 1;
  const float* acc = A.t.ACC_src[cur] + (size_t)p * n;
  const float mcur = A.t.Msrc[cur][p];
  float* S = A.S + (size_t)p * n;

  // MM step: nu_j = log w_j + (ln2 / x_j) sum_i D_ij (LA2_i - log2 S_i), LA2 = M + log2(sum)
  float accq[KQ];
#pragma unroll
  for (int q = 0; q < KQ; ++q) accq[q] = 0.f;
  for (int base = warp * 32; base < n; base += 8 * 32) {
    const int i = base + lane;
    float r = 0.f;
    if (i < n) {
      const float s = S[i];
      r = s > 0.f ? (mcur + P::log2(acc[i])) - P::log2(s) : 0.f;
    }
    const int cnt = min(32, n - base);
    for (int t = 0; t < cnt; ++t) {
      const float rt = __shfl_sync(0xffffffffu, r, t);
      const float* Drow = A.D + (size_t)(base + t) * k;
#pragma unroll
      for (int q = 0; q < KQ; ++q) {
        const int j = lane + 32 * q;
        if (j < k) accq[q] = fmaf(Drow[j], rt, accq[q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < KQ; ++q) red_s[warp][lane + 32 * q] = accq[q];
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    float sum = 0.f;
#pragma unroll
    for (int w8 = 0; w8 < 8; ++w8) sum += red_s[w8][j];
    const float xj = A.xcol[j];
    const float wold = A.W[(size_t)p * k + j];
    const float nu = P::log(wold) + sum * float(kLn2) / xj;
    float wn;
    if (A.penalty == PEN_L1) wn = P::exp(nu - A.alpha / (A.eps * xj));
    else if (A.penalty == PEN_L2SQ) {
      const float c = A.alpha / (A.eps * xj);
      wn = wright_omega<float>(P::log(c) + nu) / c;
    } else wn = P::exp(nu);
    A.W[(size_t)p * k + j] = wn;
    w_s[j] = wn;
  }
  __syncthreads();

  // source step: S = D w, F2 = log2 S - LA2, then the target operand from F2
  float* F2 = A.F2 + (size_t)p * n;
  float mass = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float s = 0.f;
    for (int j = 0; j < k; ++j) s = fmaf(A.Dt[(size_t)j * n + i], w_s[j], s);
    if (s < P::tiny()) s = 0.f;
    S[i] = s;
    const float a = acc[i];
    F2[i] = (s > 0.f) ? P::log2(s) - (mcur + P::log2(a)) : P::ninf();
    mass += s;
  }
  mass = block_sum(mass, red);
  if (threadIdx.x == 0) A.mass[p] = mass;
  __syncthreads();
  const float mt = write_operand(F2, n, A.t.ld, slot, A.t.Vhi, A.t.Vlo, red);
  if (threadIdx.x == 0) A.t.Mtgt[p] = mt;
}

// t = Q^T 1 = 2^{G2 + LB2}, LB2 = Mtgt + log2(target sum); w, g and the per-problem statistics.
__global__ void tc_finalize_kernel(FinArgs<float> F, const float* ACC_tgt, const float* Mtgt) {
  using P = Prec<float>;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t bn = (size_t)F.batch * F.n, bk = (size_t)F.batch * F.k;
  for (size_t e = tid; e < bk; e += stride) F.w_out[e] = F.W[e];
  for (size_t e = tid; e < bn; e += stride) {
    const int p = (int)(e / F.n);
    if (F.g_out) F.g_out[e] = F.G2[e] * F.gscale_inv;
    if (F.t_out) {
      const float s = ACC_tgt[e];
      F.t_out[e] = s > 0.f ? P::exp2(F.G2[e] + Mtgt[p] + P::log2(s)) : 0.f;
    }
  }
  for (size_t e = tid; e < (size_t)F.batch; e += stride) {
    if (F.iters_out) F.iters_out[e] = F.iters[e];
    if (F.status_out) F.status_out[e] = F.status[e];
    if (F.err_out) F.err_out[e] = F.err[e];
  }
}

// Run Algorithm 1 with tensor-core applies (float buffers; x, D, y, w, g as in solve_device).
// Returns cudaErrorLaunchTimeout when a GEMM reported an expired wait.
inline cudaError_t solve_device_tc(const Launch& L, const Workspace<float>& ws, const TcWorkspace& tw,
                                   const SolveParams& sp, const float* x, const float* D, const float* y, float* w,
                                   float* g, float* t_out, int* iters_out, float* err_out, int* status_out) {
  const int batch = sp.batch, n = sp.n, k = sp.k;
  const double eps_ln2 = sp.eps * kLn2;
  PrepArgs<float> pa;
  pa.x = x; pa.D = D; pa.w_in = w; pa.g_in = g; pa.y = y;
  pa.xt = ws.xt; pa.Dt = ws.Dt; pa.xcol = ws.xcol; pa.W = ws.W; pa.G2 = ws.G2;
  pa.active = ws.active; pa.done = ws.done; pa.n_active = ws.n_active; pa.err_acc = ws.err_acc;
  pa.iters = ws.iters; pa.status = ws.status; pa.err = ws.err;
  pa.batch = batch; pa.n = n; pa.k = k;
  pa.xscale = float(1.0 / sqrt(eps_ln2));
  pa.gscale = float(1.0 / eps_ln2);
  L.begin(KIND_OTHER);
  prep_kernel<float><<<1184, 256, 0, L.stream>>>(pa);
  L.end();
  L.begin(KIND_OTHER);
  colsum_kernel<float><<<(k + 7) / 8, 256, 0, L.stream>>>(ws.Dt, ws.xcol, n, k);
  L.end();
  L.begin(KIND_OTHER);
  source_init_kernel<float><<<batch, 256, 0, L.stream>>>(ws.Dt, ws.W, ws.S, ws.mass, n, k);
  L.end();
  L.begin(KIND_OTHER);
  kbuild_kernel<<<2048, 256, 0, L.stream>>>(ws.xt, n, tw.ld, tw.Khi, tw.Klo);
  L.end();
  cudaError_t e = cudaMemsetAsync(tw.err, 0, sizeof(int), L.stream);
  if (e != cudaSuccess) return e;

  TcIterArgs ta{};
  ta.active = ws.active; ta.n_active = ws.n_active; ta.n = n; ta.k = k; ta.ld = tw.ld;
  ta.max_iter = sp.max_iter; ta.datafit = sp.datafit; ta.penalty = sp.penalty;
  ta.tol = float(sp.tol); ta.eps = float(sp.eps); ta.alpha = float(sp.alpha);
  ta.kl_coef = float(sp.lam / (sp.eps + sp.lam)); ta.tv_bound = float(sp.lam / eps_ln2);
  ta.lam_over_eps = float(sp.lam / sp.eps); ta.log_lam_over_eps = float(log(sp.lam / sp.eps));
  ta.y = y; ta.D = D; ta.Dt = ws.Dt; ta.xcol = ws.xcol; ta.G2 = ws.G2; ta.S = ws.S; ta.F2 = ws.F2; ta.W = ws.W;
  ta.mass = ws.mass; ta.err = ws.err; ta.done = ws.done; ta.iters = ws.iters; ta.status = ws.status; ta.t = tw;

  tc::GemmArgs gs{nullptr, ws.active, ws.n_active, n, batch, n, n, tw.err};
  for (int it = 0;; ++it) {
    ta.it = it;
    L.begin(KIND_MM);
    tc_prep_src_kernel<<<batch, 256, 0, L.stream>>>(ta);
    L.end();
    gs.out = tw.ACC_src[it & 1];
    L.begin(KIND_APPLY);
    e = tc::launch_gemm3(tw.Khi, tw.Klo, tw.Vhi, tw.Vlo, n, batch, n, tw.ld, gs, L.stream);
    L.end();
    if (e != cudaSuccess) return e;
    if (it > 0) {
      L.begin(KIND_MM);
      tc_violation_kernel<<<batch, 256, 0, L.stream>>>(ta);
      L.end();
      L.begin(KIND_COMPACT);
      compact_kernel<<<1, 1024, 0, L.stream>>>(ws.active, ws.n_active, ws.done);
      L.end();
    }
    if (it >= sp.max_iter) break;
    L.begin(KIND_MM);
    if (k <= 32) tc_mm_kernel<1><<<batch, 256, 0, L.stream>>>(ta);
    else if (k <= 64) tc_mm_kernel<2><<<batch, 256, 0, L.stream>>>(ta);
    else if (k <= 128) tc_mm_kernel<4><<<batch, 256, 0, L.stream>>>(ta);
    else tc_mm_kernel<8><<<batch, 256, 0, L.stream>>>(ta);
    L.end();
    gs.out = tw.ACC_tgt;
    L.begin(KIND_APPLY);
    e = tc::launch_gemm3(tw.Khi, tw.Klo, tw.Vhi, tw.Vlo, n, batch, n, tw.ld, gs, L.stream);
    L.end();
    if (e != cudaSuccess) return e;
    if ((it + 1) % sp.poll_every == 0) {
      e = cudaMemcpyAsync(L.host_flag, ws.n_active, sizeof(int), cudaMemcpyDeviceToHost, L.stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
      if (e == cudaSuccess && L.timer && L.timer->on) e = L.timer->harvest();
      if (e != cudaSuccess) return e;
      if (*L.host_flag == 0) break;
    }
  }
  FinArgs<float> fa;
  fa.W = ws.W; fa.G2 = ws.G2; fa.LB2 = nullptr; fa.iters = ws.iters; fa.status = ws.status; fa.err = ws.err;
  fa.w_out = w; fa.g_out = g; fa.t_out = t_out; fa.iters_out = iters_out; fa.status_out = status_out;
  fa.err_out = err_out; fa.batch = batch; fa.n = n; fa.k = k; fa.gscale_inv = float(eps_ln2);
  L.begin(KIND_OTHER);
  tc_finalize_kernel<<<1184, 256, 0, L.stream>>>(fa, tw.ACC_tgt, tw.Mtgt);
  L.end();
  e = cudaMemcpyAsync(L.host_flag, tw.err, sizeof(int), cudaMemcpyDeviceToHost, L.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
  if (e == cudaSuccess && L.timer && L.timer->on) e = L.timer->harvest();
  if (e != cudaSuccess) return e;
  return *L.host_flag ? cudaErrorLaunchTimeout : cudaGetLastError();
}

}  // namespace otlm
