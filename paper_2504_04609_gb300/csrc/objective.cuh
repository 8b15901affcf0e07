// otlm_objective: objective and Fenchel dual of a caller's state (w, g), reduced in FP64 with the
// kernels of objective_kernels.cuh; the applies run in the handle's FP32 / FP64 arithmetic.
#pragma once

#include "objective_kernels.cuh"
#include "solver.cuh"

namespace otlm {

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
  pa.dw = ws.dw; pa.all = ws.all; pa.all_count = ws.all_count;
  pa.batch = batch; pa.n = n; pa.k = k;
  pa.xscale = T(grid_scale(sp.cost, eps_ln2));
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
  launch_apply<T, EPI_SOURCE>(L, src, true, batch, n, sp.cost);
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
  launch_apply<T, EPI_TARGET>(L, tgt, true, batch, n, sp.cost);

  // sum(K) in FP64
  double* kmass = ws.kmass;
  cudaError_t e = cudaMemsetAsync(kmass, 0, sizeof(double), L.stream);
  if (e != cudaSuccess) return e;
  L.begin(KIND_OTHER);
  kernel_mass_kernel<T><<<592, 256, 0, L.stream>>>(x, n, 1.0 / sp.eps, kmass, sp.cost == COST_ABS);
  L.end();

  ObjArgs<T> oa{};
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
