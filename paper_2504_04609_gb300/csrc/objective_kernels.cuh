// Kernels of the objective and Fenchel dual of a solver state (w, g), reduced in FP64 (Eq. OTLM, reading with
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
//   L2 sum(-g'y + g'^2/(2 lam)) where y - g'/lam >= 0, else -lam y^2 / 2; balanced -<g', y>;
//   Poisson (reading A7) sum_{y>0} lam y (log(lam y / (lam + g')) - 1), finite for g' > -lam.  The
//   datafit step gives lam + g' = lam y / v' with v' = 2^(G2' + LB2) (the prox value), so the dual
//   takes g' = lam y / v' - lam in FP64 (and -lam where y = 0): a dual-feasible point whose
//   conjugate term is lam y (log v' - 1), free of the cancellation in lam + g' that FP32
//   potentials cannot resolve at small y.
// A row whose source mass underflowed (s_i = 0) under a non-zero dictionary row enters D^T f with
// the smallest finite f instead of -inf.
#pragma once

#include "kernels.cuh"

namespace otlm {

// sum_ij exp(-C_ij / eps) of the grid cost ((x_i - x_j)^2, or |x_i - x_j| when abs_cost) in FP64,
// accumulated into *out (zeroed by the caller).
template <typename T>
__global__ void kernel_mass_kernel(const T* x, int n, double inv_eps, double* out, int abs_cost) {
  __shared__ double red[32];
  double acc = 0.0;
  const size_t nn = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / n, j = e - i * n;
    const double d = (double)x[i] - (double)x[j];
    acc += ::exp(-(abs_cost ? ::fabs(d) : d * d) * inv_eps);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}

// sum_ij exp(-C_ij / eps) for a dense cost C [n][n] (+inf allowed) in FP64.
template <typename T>
__global__ void kernel_mass_dense_kernel(const T* C, int n, double inv_eps, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  const size_t nn = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x)
    acc += ::exp(-(double)C[e] * inv_eps);
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}

// F2 = log2 S - LA2 (-inf where S = 0) of the listed problems: the source potential of the state
// (w, g) whose a = K u1 is in LA2 and whose s = D w is in S (one CTA per listed problem).
template <typename T>
__global__ void obj_f2_kernel(const int* list, const int* count, const T* S, const T* LA2, T* F2, int n) {
  using P = Prec<T>;
  if ((int)blockIdx.x >= *count) return;
  const size_t o = (size_t)list[blockIdx.x] * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const T s = S[o + i];
    F2[o + i] = s > T(0) ? P::log2(s) - LA2[o + i] : P::ninf();
  }
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
  const int* list;     // problems to evaluate (CTA b takes list[b] while b < *count); null: p = b
  const int* count;
  int* gap_ok;         // when not null: gap_ok[p] = (primal - dual <= gap_tol |primal|)
  double gap_tol;
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
  if (A.list && (int)blockIdx.x >= *A.count) return;
  const int p = A.list ? A.list[blockIdx.x] : (int)blockIdx.x;
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
      case DF_POISSON:
        L += yv > 0.0 ? t - yv * ::log(t) : t;
        if (yv > 0.0) {
          // g' = lam y / v' - lam (see the header); its entropic term replaces the one above
          const double v = ::exp2((double)G2n[j] + lb);
          f2c += A.lam * yv * (::log(v) - 1.0);
          const double gp = A.lam * yv / v - A.lam;
          vsum += ::exp2(gp / el2 + lb) - v;
        }
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

  // D^T f, k <= 256 columns, one column per thread, rows in sequence.  FP32 element types take
  // each product exactly as a float pair (fma gives the rounding error of d * F2) and add it with a
  // two-sum into a float pair, moved into an FP64 sum every 64 rows: FP64-grade accuracy without
  // an FP64 multiply-add per dictionary entry (the FP64 pipe is the slow one here).
  const double f2_lo = f_lo / el2;  // log2 units
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double acc = 0.0;
    if constexpr (sizeof(T) == 4) {
      for (int i0 = 0; i0 < n; i0 += 64) {
        float hi = 0.f, lo = 0.f;
        const int i1 = min(n, i0 + 64);
        for (int i = i0; i < i1; ++i) {
          const float d = (float)A.D[(size_t)i * k + j];
          if (d > 0.f) {
            float fv = (float)F2[i];
            if (!isfinite(fv)) fv = (float)f2_lo;
            const float pr = d * fv, pe = fmaf(d, fv, -pr);
            const float s = hi + pr, bb = s - hi;
            lo += (hi - (s - bb)) + (pr - bb) + pe;
            hi = s;
          }
        }
        acc += (double)hi + (double)lo;
      }
      acc *= el2;
    } else {
      for (int i = 0; i < n; ++i) {
        const double d = A.D[(size_t)i * k + j];
        if (d > 0.0) {
          double f = el2 * (double)F2[i];
          if (!isfinite(f)) f = f_lo;
          acc += d * f;
        }
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
    const double P = sf + tg - A.eps * ssum + A.eps * kmass + datafit_term + R;
    const double Dv = -f1c - f2c - A.eps * (::exp(c / A.eps) * vsum - kmass);
    A.primal[p] = P;
    A.dual[p] = Dv;
    if (A.gap_ok) A.gap_ok[p] = (P - Dv <= A.gap_tol * fabs(P)) ? 1 : 0;
  }
}

}  // namespace otlm
