// Objective and Fenchel dual of a solver state (w, g), reduced in FP64 (Eq. OTLM, reading with
// the objective eps KL(Q||K) + lam L(Q^T 1|y) + alpha R(w)).
//
// From (w, g): a = K u1, s = D w, f = eps log(s/a) gives the plan Q = diag(e^{f/eps}) K diag(e^{g/eps})
// with Q 1 = s = D w (feasible), t = Q^T 1 = u1 * K^T u2, and
//   eps KL(Q||K) = <f, s> + <g, t> - eps sum(s) + eps sum(K).
// Dual at (f', g'):  -F1*(-f') - F2*(-g') - eps (sum_ij K_ij e^{(f'_i + g'_j)/eps} - sum(K)), with
//   g' = the datafit step from b = K^T u2 (the g the next iteration would use), and
//   f' = f + c 1, c >= 0 the smallest shift with D^T f' >= -alpha (l1) or >= 0 (no penalty), so
//   sum_ij K e^{(f'+g')/eps} = e^{c/eps} sum_j 2^(G2'_j + LB2_j).
//   F1*(-f') = sum_j max(-(D^T f)_j, 0)^2 / (2 alpha) for the squared-l2 penalty, 0 otherwise.
//   F2*(-g') per datafit: KL lam sum y (e^{-g'/lam} - 1); TV -sum y min(g', lam);
//   L2 sum(-g'y + g'^2/(2 lam)) where y - g'/lam >= 0, else -lam y^2 / 2; balanced -<g', y>.
// A row whose source mass underflowed (s_i = 0) under a non-zero dictionary row enters D^T f with
// the smallest finite f instead of -inf.
#pragma once

#include "kernels.cuh"
#include "solver.cuh"

namespace otlm {

// sum_ij exp(-(x_i - x_j)^2 / eps) in FP64, accumulated into *out (zeroed by the caller).
template <typename T>
__global__ void kernel_mass_kernel(const T* x, int n, double inv_eps, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  const size_t nn = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / n, j = e - i * n;
    const double d = (double)x[i] - (double)x[j];
    acc += ::exp(-d * d * inv_eps);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}

template <typename T>
__global__ void objective_source_kernel(const T* Dt, const T* W, const T* LA2, T* S, T* F2, T* mass, int n, int k) {
  __shared__ T w_s[256];
  __shared__ T red[32];
  const int p = blockIdx.x;
  for (int j = threadIdx.x; j < k; j += blockDim.x) w_s[j] = W[(size_t)p * k + j];
  __syncthreads();
  const T m = source_marginal<T>(Dt, w_s, n, k, S + (size_t)p * n, F2 + (size_t)p * n, LA2 + (size_t)p * n, red);
  if (threadIdx.x == 0) mass[p] = m;
}

template <typename T>
struct ObjArgs {
  const T* D; const T* xcol; const T* W; const T* y;
  const T* S; const T* F2; const T* G2; const T* LB2; const T* G2n;
  const double* kmass;
  double* primal; double* dual;
  int n, k, datafit, penalty;
  double eps, lam, alpha, beta, balanced_rtol;
};

__device__ __forceinline__ double block_min(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : CUDART_INF;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (threadIdx.x == 0) red[0] = v;
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

// One CTA (256 threads) per problem.
template <typename T>
__global__ void __launch_bounds__(256) objective_reduce_kernel(ObjArgs<T> A) {
  __shared__ double red[32];
  __shared__ double xtf_s[256];
  const int p = blockIdx.x;
  const int n = A.n, k = A.k;
  const double el2 = A.eps * kLn2;
  const T* S = A.S + (size_t)p * n;
  const T* F2 = A.F2 + (size_t)p * n;
  const T* G2 = A.G2 + (size_t)p * n;
  const T* LB2 = A.LB2 + (size_t)p * n;
  const T* G2n = A.G2n + (size_t)p * n;
  const T* y = A.y + (size_t)p * n;

  // source side: <f, s>, sum s, smallest finite f
  double sf = 0.0, ssum = 0.0, f_lo = CUDART_INF;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double s = S[i];
    const double f = el2 * (double)F2[i];
    if (s > 0.0) {
      sf += s * f;
      ssum += s;
    }
    if (isfinite(f)) f_lo = f_lo < f ? f_lo : f;
  }
  sf = block_sum(sf, red);
  ssum = block_sum(ssum, red);
  f_lo = block_min(f_lo, red);

  // target side: <g, t>, datafit value, F2*(-g'), sum_j v'_j
  double tg = 0.0, L = 0.0, f2c = 0.0, vsum = 0.0, bal_dev = 0.0, ymax = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double lb = LB2[j];
    const double t = ::exp2((double)G2[j] + lb);
    const double gv = el2 * (double)G2[j];
    const double yv = (double)y[j] >= (double)Prec<T>::tiny() ? (double)y[j] : 0.0;  // FTZ, as the applies
    const double gn = el2 * (double)G2n[j];
    if (t > 0.0) tg += t * gv;
    vsum += ::exp2((double)G2n[j] + lb);
    switch (A.datafit) {
      case DF_KL:
        L += (t > 0.0 ? t * ::log(t / yv) : 0.0) - t + yv;
        if (yv > 0.0) f2c += A.lam * yv * ::expm1(-gn / A.lam);
        break;
      case DF_TV:
        L += fabs(t - yv);
        f2c += -yv * fmin(gn, A.lam);
        break;
      case DF_L2:
        L += 0.5 * (t - yv) * (t - yv);
        f2c += (yv - gn / A.lam >= 0.0) ? (-gn * yv + gn * gn / (2.0 * A.lam)) : (-A.lam * yv * yv * 0.5);
        break;
      default:
        bal_dev = fmax(bal_dev, fabs(t - yv));
        ymax = fmax(ymax, yv);
        if (yv > 0.0) f2c += -gn * yv;  // a bin with y = 0 contributes 0 whatever g is
    }
  }
  tg = block_sum(tg, red);
  vsum = block_sum(vsum, red);
  L = block_sum(L, red);
  f2c = block_sum(f2c, red);
  bal_dev = block_max(bal_dev, red);
  ymax = block_max(ymax, red);

  // D^T f (FP64), k <= 256 columns, one column per thread, rows in sequence
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
      const double d = A.D[(size_t)i * k + j];
      if (d > 0.0) {
        double f = el2 * (double)F2[i];
        if (!isfinite(f)) f = f_lo;
        acc += d * f;
      }
    }
    xtf_s[j] = acc;
  }
  __syncthreads();

  // weighted penalty, F1* and the feasibility shift c
  double R = 0.0, f1c = 0.0, c = 0.0;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double wj = A.W[(size_t)p * k + j];
    const double xtf = xtf_s[j];
    if (A.penalty == PEN_L1) {
      R += A.alpha * wj;
      c = fmax(c, (-A.alpha - xtf) / (double)A.xcol[j]);
    } else if (A.penalty == PEN_L2SQ) {
      R += 0.5 * A.alpha * wj * wj;
      const double v = fmax(-xtf, 0.0);
      f1c += v * v / (2.0 * A.alpha);
    } else if (A.penalty == PEN_ELASTIC) {
      // sup_{w >= 0} (v w - alpha w - beta w^2 / 2) = (v - alpha)+^2 / (2 beta), v = -(X^T f)_j
      R += A.alpha * wj + 0.5 * A.beta * wj * wj;
      const double v = fmax(-xtf - A.alpha, 0.0);
      f1c += v * v / (2.0 * A.beta);
    } else {
      c = fmax(c, -xtf / (double)A.xcol[j]);
    }
  }
  R = block_sum(R, red);
  f1c = block_sum(f1c, red);
  c = block_max(c, red);

  if (threadIdx.x == 0) {
    const double kmass = *A.kmass;
    double datafit_term;
    if (A.datafit == DF_BALANCED) datafit_term = (bal_dev <= A.balanced_rtol * ymax) ? 0.0 : CUDART_INF;
    else datafit_term = A.lam * L;
    A.primal[p] = sf + tg - A.eps * ssum + A.eps * kmass + datafit_term + R;
    A.dual[p] = -f1c - f2c - A.eps * (::exp(c / A.eps) * vsum - kmass);
  }
}

template <typename T>
cudaError_t objective_device(const Launch& L, const Workspace<T>& ws, const SolveParams& sp, const T* x, const T* D,
                             const T* y, const T* w, const T* g, double* primal, double* dual) {
  const int batch = sp.batch, n = sp.n, k = sp.k;
  const double eps_ln2 = sp.eps * kLn2;
  PrepArgs<T> pa;
  pa.x = x; pa.D = D; pa.w_in = w; pa.g_in = g; pa.y = y;
  pa.xt = ws.xt; pa.Dt = ws.Dt; pa.xcol = ws.xcol; pa.W = ws.W; pa.G2 = ws.G2;
  pa.active = ws.active; pa.done = ws.done; pa.n_active = ws.n_active; pa.err_acc = ws.err_acc;
  pa.iters = ws.iters; pa.status = ws.status; pa.err = ws.err;
  pa.batch = batch; pa.n = n; pa.k = k;
  pa.xscale = T(1.0 / sqrt(eps_ln2));
  pa.gscale = T(1.0 / eps_ln2);
  L.begin(KIND_OTHER);
  prep_kernel<T><<<1184, 256, 0, L.stream>>>(pa);
  L.end();
  L.begin(KIND_OTHER);
  colsum_kernel<T><<<(k + 7) / 8, 256, 0, L.stream>>>(ws.Dt, ws.xcol, n, k);
  L.end();

  // a = K u1, then s = D w and f
  ApplyArgs<T> src{};
  src.in = ws.G2; src.out = ws.LA2; src.xt = ws.xt; src.active = ws.active; src.n_active = ws.n_active;
  src.n = n; src.S = ws.S; src.err_acc = ws.err_acc; src.check = 0;
  launch_apply<T, EPI_SOURCE>(L, src, true, batch, n);
  L.begin(KIND_OTHER);
  objective_source_kernel<T><<<batch, 256, 0, L.stream>>>(ws.Dt, ws.W, ws.LA2, ws.S, ws.F2, ws.mass, n, k);
  L.end();

  // b = K^T u2 and the datafit step g' (written over LA2, which is no longer needed)
  ApplyArgs<T> tgt = src;
  tgt.in = ws.F2; tgt.out = ws.LB2; tgt.y = y; tgt.G2 = ws.LA2; tgt.datafit = sp.datafit;
  tgt.kl_coef = T(sp.lam / (sp.eps + sp.lam));
  tgt.tv_bound = T(sp.lam / eps_ln2);
  tgt.lam_over_eps = T(sp.lam / sp.eps);
  tgt.log_lam_over_eps = T(log(sp.lam / sp.eps));
  launch_apply<T, EPI_TARGET>(L, tgt, true, batch, n);

  // sum(K) in FP64
  double* kmass = ws.kmass;
  cudaError_t e = cudaMemsetAsync(kmass, 0, sizeof(double), L.stream);
  if (e != cudaSuccess) return e;
  L.begin(KIND_OTHER);
  kernel_mass_kernel<T><<<592, 256, 0, L.stream>>>(x, n, 1.0 / sp.eps, kmass);
  L.end();

  ObjArgs<T> oa;
  oa.D = D; oa.xcol = ws.xcol; oa.W = ws.W; oa.y = y; oa.S = ws.S; oa.F2 = ws.F2; oa.G2 = ws.G2; oa.LB2 = ws.LB2;
  oa.G2n = ws.LA2; oa.kmass = kmass; oa.primal = primal; oa.dual = dual; oa.n = n; oa.k = k;
  oa.datafit = sp.datafit; oa.penalty = sp.penalty; oa.eps = sp.eps; oa.lam = sp.lam; oa.alpha = sp.alpha; oa.beta = sp.beta;
  oa.balanced_rtol = sizeof(T) == 4 ? 1e-4 : 1e-10;
  L.begin(KIND_OTHER);
  objective_reduce_kernel<T><<<batch, 256, 0, L.stream>>>(oa);
  L.end();
  e = cudaGetLastError();
  if (e == cudaSuccess && L.timer && L.timer->on) e = L.timer->harvest();
  return e;
}

}  // namespace otlm
