// Host driver of the batched scaling iteration: workspace layout and the per-iteration launch
// sequence (source apply -> MM/source step -> compaction -> target apply/prox), for one precision.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "kernels.cuh"
#include "objective_kernels.cuh"

namespace otlm {

// Optional device timing of launches by kind: each launch is bracketed by two events on the
// launching stream; pairs are harvested at the host's convergence polls and at the end of a solve.
enum { KIND_APPLY = 0, KIND_MM = 1, KIND_COMPACT = 2, KIND_OTHER = 3, KIND_COUNT = 4 };

struct Timer {
  static constexpr int kPairs = 96;
  bool on = false;
  cudaEvent_t ev[2 * kPairs];
  int kind[kPairs];
  int used = 0;
  double ms[KIND_COUNT] = {0, 0, 0, 0};
  long long count[KIND_COUNT] = {0, 0, 0, 0};

  cudaError_t create() {
    for (int i = 0; i < 2 * kPairs; ++i) {
      cudaError_t e = cudaEventCreate(&ev[i]);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  void destroy() {
    for (int i = 0; i < 2 * kPairs; ++i) cudaEventDestroy(ev[i]);
  }
  // Sum the recorded pairs; the caller has synchronised the stream (or we wait here).
  cudaError_t harvest() {
    for (int i = 0; i < used; ++i) {
      float t = 0.f;
      cudaError_t e = cudaEventSynchronize(ev[2 * i + 1]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
      if (e != cudaSuccess) return e;
      ms[kind[i]] += t;
      count[kind[i]] += 1;
    }
    used = 0;
    return cudaSuccess;
  }
};

struct Launch {
  cudaStream_t stream;
  long long* counter;
  int* host_flag;  // pinned int used for the convergence polls
  Timer* timer;    // may be null

  // Bracket one launch: call begin(kind) before and end() after it.
  void begin(int k) const {
    if (timer && timer->on) {
      if (timer->used == Timer::kPairs) timer->harvest();
      timer->kind[timer->used] = k;
      cudaEventRecord(timer->ev[2 * timer->used], stream);
    }
  }
  void end() const {
    ++*counter;
    if (timer && timer->on) {
      cudaEventRecord(timer->ev[2 * timer->used + 1], stream);
      ++timer->used;
    }
  }
};

template <typename T>
struct Workspace {
  T *xt, *Dt, *xcol, *G2, *LA2, *LB2, *F2, *S, *W, *mass, *err_acc, *err;
  T* dw;      // [batch] ||dw||_1 / ||w||_1 of the last MM update
  T* Wprev;   // [batch][k] weights before the last update (tensor-core path)
  int *active, *n_active, *done, *iters, *status;
  int *all, *all_count;  // every problem of the batch, in order (the final objective's list)
  double* kmass;
};

// Scratch of the in-solve objective (handles created with check_every > 0): the state's source
// potential, its target sums and datafit step, and the per-problem FP64 primal, dual and gap test.
template <typename T>
struct ObjWorkspace {
  T* F2;          // [batch][n]
  T* LB2;         // [batch][n] (tensor-core path: the raw target sums first, decoded in place)
  T* G2n;         // [batch][n]
  T* M;           // [batch] target shift of the tensor-core operand
  double *primal, *dual;  // [batch]
  int* gap_ok;    // [batch]
  double* kmass;  // sum_ij K_ij
};

inline size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

// Bytes of one workspace for the given maxima, and the carving of a base pointer into it.
template <typename T>
size_t carve_workspace(void* base, int n_max, int k_max, int batch_max, Workspace<T>* ws) {
  const size_t bn = (size_t)batch_max * n_max, bk = (size_t)batch_max * k_max;
  size_t off = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* p = b ? b + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  Workspace<T> w;
  w.xt = (T*)take(sizeof(T) * n_max);
  w.Dt = (T*)take(sizeof(T) * (size_t)n_max * k_max);
  w.xcol = (T*)take(sizeof(T) * k_max);
  w.G2 = (T*)take(sizeof(T) * bn);
  w.LA2 = (T*)take(sizeof(T) * bn);
  w.LB2 = (T*)take(sizeof(T) * bn);
  w.F2 = (T*)take(sizeof(T) * bn);
  w.S = (T*)take(sizeof(T) * bn);
  w.W = (T*)take(sizeof(T) * bk);
  w.mass = (T*)take(sizeof(T) * batch_max);
  w.err_acc = (T*)take(sizeof(T) * batch_max);
  w.err = (T*)take(sizeof(T) * batch_max);
  w.dw = (T*)take(sizeof(T) * batch_max);
  w.Wprev = (T*)take(sizeof(T) * bk);
  w.all = (int*)take(sizeof(int) * batch_max);
  w.all_count = (int*)take(sizeof(int) * 32);
  w.active = (int*)take(sizeof(int) * batch_max);
  w.n_active = (int*)take(sizeof(int) * 32);
  w.done = (int*)take(sizeof(int) * batch_max);
  w.iters = (int*)take(sizeof(int) * batch_max);
  w.status = (int*)take(sizeof(int) * batch_max);
  w.kmass = (double*)take(sizeof(double) * 4);
  if (ws) *ws = w;
  return off;
}

template <typename T>
size_t carve_obj_workspace(void* base, int n_max, int batch_max, ObjWorkspace<T>* ow) {
  const size_t bn = (size_t)batch_max * n_max;
  size_t off = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* p = b ? b + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  ObjWorkspace<T> o;
  o.F2 = (T*)take(sizeof(T) * bn);
  o.LB2 = (T*)take(sizeof(T) * bn);
  o.G2n = (T*)take(sizeof(T) * bn);
  o.M = (T*)take(sizeof(T) * batch_max);
  o.primal = (double*)take(sizeof(double) * batch_max);
  o.dual = (double*)take(sizeof(double) * batch_max);
  o.gap_ok = (int*)take(sizeof(int) * batch_max);
  o.kmass = (double*)take(sizeof(double) * 4);
  if (ow) *ow = o;
  return off;
}

struct SolveParams {
  int batch, n, k;
  double eps, lam, alpha;
  int datafit, penalty, max_iter, poll_every;
  double tol;
  double beta = 0.0;  // elastic net's squared-l2 weight
  int mm_steps = 1;   // MM steps per iteration
  int check_every = 0;   // FP64 objective / gap every this many iterations and at the end (0: never)
  double gap_tol = 0.0;  // stop also requires (primal - dual) <= gap_tol |primal| at a check
  double dw_tol = 0.0;   // stop also requires ||dw||_1 / ||w||_1 <= dw_tol
  double single_until = 0.0;  // tensor cores: single BF16 product until a violation is <= this
  int cost = COST_SQ;         // grid cost: COST_SQ (x_i - x_j)^2 or COST_ABS |x_i - x_j|
};

// Scale of the grid that turns the cost into log2 units: (xt_i - xt_j)^2 = (x_i - x_j)^2 / (eps ln2)
// or |xt_i - xt_j| = |x_i - x_j| / (eps ln2).
inline double grid_scale(int cost, double eps_ln2) {
  return cost == COST_ABS ? 1.0 / eps_ln2 : 1.0 / sqrt(eps_ln2);
}

// Argument block of the FP64 reduction for a state held in the workspaces (S, G2, the weights)
// with its source potential, target sums and datafit step in the objective scratch.
template <typename T>
ObjArgs<T> obj_args(const SolveParams& sp, const T* D, const T* xcol, const T* W, const T* y, const T* S,
                    const T* G2, const ObjWorkspace<T>& ow) {
  ObjArgs<T> oa{};
  oa.D = D; oa.xcol = xcol; oa.W = W; oa.y = y; oa.S = S; oa.F2 = ow.F2; oa.G2 = G2; oa.LB2 = ow.LB2;
  oa.G2n = ow.G2n; oa.kmass = ow.kmass; oa.primal = ow.primal; oa.dual = ow.dual; oa.n = sp.n; oa.k = sp.k;
  oa.datafit = sp.datafit; oa.penalty = sp.penalty; oa.eps = sp.eps; oa.lam = sp.lam; oa.alpha = sp.alpha;
  oa.beta = sp.beta; oa.balanced_rtol = sizeof(T) == 4 ? 1e-4 : 1e-10; oa.gap_tol = sp.gap_tol;
  return oa;
}

template <typename T> struct TileFor;
// FP32 apply tile (problems per thread, rows per thread, warps along problems, warps along rows,
// columns per staged chunk); chosen by the tile sweep recorded in profiles/.
#ifndef OTLM_F32_RB
#define OTLM_F32_RB 4
#endif
#ifndef OTLM_F32_RI
#define OTLM_F32_RI 4
#endif
#ifndef OTLM_F32_WB
#define OTLM_F32_WB 4
#endif
#ifndef OTLM_F32_TJ
#define OTLM_F32_TJ 64
#endif
template <> struct TileFor<float> {
  using type = ApplyTile<float, OTLM_F32_RB, OTLM_F32_RI, OTLM_F32_WB, 1, OTLM_F32_TJ>;
  // small batches x grids: half the rows per CTA, twice the CTAs, half the accumulators per thread
  using small = ApplyTile<float, OTLM_F32_RB, OTLM_F32_RI / 2, OTLM_F32_WB, 1, OTLM_F32_TJ>;
};
template <> struct TileFor<double> { using type = ApplyTile<double, 2, 2, 2, 2, 32>; };

// first = true: no previous sums exist yet, shift by the diagonal term.
inline int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 152;
  }
  return sms;
}

template <typename T, typename Cfg, int EPI>
void launch_apply_cfg(const Launch& L, const ApplyArgs<T>& a, bool first, int batch, int n, int cost) {
  const dim3 grid((n + Cfg::TI - 1) / Cfg::TI, (batch + Cfg::TB - 1) / Cfg::TB);
  L.begin(KIND_APPLY);
  if (a.C) {
    if (first) apply_kernel<T, Cfg, EPI, SHIFT_DIAG, COST_DENSE><<<grid, Cfg::NT, 0, L.stream>>>(a);
    else apply_kernel<T, Cfg, EPI, SHIFT_PREV, COST_DENSE><<<grid, Cfg::NT, 0, L.stream>>>(a);
  } else if (cost == COST_ABS) {
    if (first) apply_kernel<T, Cfg, EPI, SHIFT_DIAG, COST_ABS><<<grid, Cfg::NT, 0, L.stream>>>(a);
    else apply_kernel<T, Cfg, EPI, SHIFT_PREV, COST_ABS><<<grid, Cfg::NT, 0, L.stream>>>(a);
  } else {
    if (first) apply_kernel<T, Cfg, EPI, SHIFT_DIAG, COST_SQ><<<grid, Cfg::NT, 0, L.stream>>>(a);
    else apply_kernel<T, Cfg, EPI, SHIFT_PREV, COST_SQ><<<grid, Cfg::NT, 0, L.stream>>>(a);
  }
  L.end();
}

// The FP32 apply takes the half-height tile when the default tile would give fewer than eight CTAs
// per SM (at n = 1024 x 1024 problems it gives 512 CTAs, 3.4 per SM at four resident: a quarter of
// the warps the exponent unit needs to stay busy).
template <typename T, int EPI>
void launch_apply(const Launch& L, const ApplyArgs<T>& a, bool first, int batch, int n, int cost) {
  using Cfg = typename TileFor<T>::type;
  if constexpr (sizeof(T) == 4) {
    const long long ctas = (long long)((n + Cfg::TI - 1) / Cfg::TI) * ((batch + Cfg::TB - 1) / Cfg::TB);
    if (ctas < 8LL * sm_count()) {
      launch_apply_cfg<T, typename TileFor<T>::small, EPI>(L, a, first, batch, n, cost);
      return;
    }
  }
  launch_apply_cfg<T, Cfg, EPI>(L, a, first, batch, n, cost);
}

template <typename T>
void launch_mm(const Launch& L, const MMArgs<T>& a, int batch) {
  L.begin(KIND_MM);
  if (a.k <= 32) mm_kernel<T, 1><<<batch, 256, 0, L.stream>>>(a);
  else if (a.k <= 64) mm_kernel<T, 2><<<batch, 256, 0, L.stream>>>(a);
  else if (a.k <= 128) mm_kernel<T, 4><<<batch, 256, 0, L.stream>>>(a);
  else mm_kernel<T, 8><<<batch, 256, 0, L.stream>>>(a);
  L.end();
}

// FP64 objective and dual (Eq. OTLM, reading A1) of the listed problems' states (w, g) from the
// a = K u1 already in LA2 and the s = D w in S: F2 = log2 s - log2 a, one target apply of F2 into
// the scratch (its datafit step g' into G2n), then the reduction; gap = true also records the gap
// test.  One extra kernel apply beside the solve's own.
template <typename T>
void objective_eval(const Launch& L, const Workspace<T>& ws, const ObjWorkspace<T>& ow, const SolveParams& sp,
                    const ApplyArgs<T>& tgt, const T* D, const T* y, const int* list, const int* count, bool gap) {
  L.begin(KIND_OTHER);
  obj_f2_kernel<T><<<sp.batch, 256, 0, L.stream>>>(list, count, ws.S, ws.LA2, ow.F2, sp.n);
  L.end();
  ApplyArgs<T> t = tgt;
  t.in = ow.F2; t.out = ow.LB2; t.G2 = ow.G2n; t.active = list; t.n_active = count; t.check = 0;
  launch_apply<T, EPI_TARGET>(L, t, true, sp.batch, sp.n, sp.cost);
  ObjArgs<T> oa = obj_args<T>(sp, D, ws.xcol, ws.W, y, ws.S, ws.G2, ow);
  oa.list = list; oa.count = count; oa.gap_ok = gap ? ow.gap_ok : nullptr;
  L.begin(KIND_OTHER);
  objective_reduce_kernel<T><<<sp.batch, 256, 0, L.stream>>>(oa);
  L.end();
}

// Run Algorithm 1 on device buffers.  Returns cudaSuccess or the first launch/copy error.
// ow (may be null when sp.check_every == 0): the objective scratch of the gap checks.
template <typename T>
cudaError_t solve_device(const Launch& L, const Workspace<T>& ws, const ObjWorkspace<T>* ow, const SolveParams& sp,
                         const T* x, const T* D, const T* y, T* w, T* g, T* t_out, int* iters_out, T* err_out,
                         int* status_out, const T* C = nullptr) {
  const int batch = sp.batch, n = sp.n, k = sp.k;
  const double eps_ln2 = sp.eps * kLn2;
  const bool checks = ow && sp.check_every > 0;

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
  L.begin(KIND_OTHER);
  source_init_kernel<T><<<batch, 256, 0, L.stream>>>(ws.Dt, ws.W, ws.S, ws.mass, n, k);
  L.end();
  if (checks) {  // sum_ij K_ij, FP64, once per solve
    cudaError_t e = cudaMemsetAsync(ow->kmass, 0, sizeof(double), L.stream);
    if (e != cudaSuccess) return e;
    L.begin(KIND_OTHER);
    if (C) kernel_mass_dense_kernel<T><<<592, 256, 0, L.stream>>>(C, n, 1.0 / sp.eps, ow->kmass);
    else kernel_mass_kernel<T><<<592, 256, 0, L.stream>>>(x, n, 1.0 / sp.eps, ow->kmass, sp.cost == COST_ABS);
    L.end();
  }

  ApplyArgs<T> src{};
  src.in = ws.G2; src.out = ws.LA2; src.xt = ws.xt; src.active = ws.active; src.n_active = ws.n_active;
  src.n = n; src.S = ws.S; src.err_acc = ws.err_acc;
  src.C = C; src.c_scale = T(1.0 / eps_ln2); src.c_trans = 0;  // dense cost (or none: the grid)
  ApplyArgs<T> tgt = src;
  tgt.c_trans = 1;
  tgt.in = ws.F2; tgt.out = ws.LB2; tgt.check = 0; tgt.y = y; tgt.G2 = ws.G2; tgt.datafit = sp.datafit;
  tgt.kl_coef = T(sp.lam / (sp.eps + sp.lam));
  tgt.tv_bound = T(sp.lam / eps_ln2);
  tgt.lam_over_eps = T(sp.lam / sp.eps);
  tgt.log_lam_over_eps = T(log(sp.lam / sp.eps));

  MMArgs<T> mm{};
  mm.active = ws.active; mm.n_active = ws.n_active; mm.n = n; mm.k = k; mm.D = D; mm.Dt = ws.Dt;
  mm.xcol = ws.xcol; mm.LA2 = ws.LA2; mm.S = ws.S; mm.F2 = ws.F2; mm.W = ws.W; mm.mass = ws.mass;
  mm.err_acc = ws.err_acc; mm.err = ws.err; mm.done = ws.done; mm.iters = ws.iters; mm.status = ws.status;
  mm.max_iter = sp.max_iter; mm.tol = T(sp.tol); mm.penalty = sp.penalty; mm.eps = T(sp.eps);
  mm.alpha = T(sp.alpha); mm.beta = T(sp.beta); mm.mm_steps = sp.mm_steps;
  mm.dw = ws.dw; mm.dw_tol = T(sp.dw_tol); mm.gap_on = checks && sp.gap_tol > 0;
  mm.gap_ok = checks ? ow->gap_ok : nullptr;

  for (int it = 0;; ++it) {
    src.check = it > 0;
    launch_apply<T, EPI_SOURCE>(L, src, it == 0, batch, n, sp.cost);
    // a check: the state (w, g) whose a = K u1 was just computed is the one this iteration returns
    // if it stops here; its FP64 objective and gap come before the stopping decision
    const bool check = checks && it > 0 && it % sp.check_every == 0;
    if (check) objective_eval<T>(L, ws, *ow, sp, tgt, D, y, ws.active, ws.n_active, true);
    mm.it = it;
    mm.gap_check = check;
    launch_mm<T>(L, mm, batch);
    L.begin(KIND_COMPACT);
    compact_kernel<<<1, 1024, 0, L.stream>>>(ws.active, ws.n_active, ws.done);
    L.end();
    if (it >= sp.max_iter) break;
    launch_apply<T, EPI_TARGET>(L, tgt, it == 0, batch, n, sp.cost);
    if ((it + 1) % sp.poll_every == 0) {
      cudaError_t e = cudaMemcpyAsync(L.host_flag, ws.n_active, sizeof(int), cudaMemcpyDeviceToHost, L.stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
      if (e == cudaSuccess && L.timer && L.timer->on) e = L.timer->harvest();
      if (e != cudaSuccess) return e;
      if (*L.host_flag == 0) break;
    }
  }

  // the returned states' objective: for every problem LA2 holds a = K u1 of its final g (computed
  // at the iteration it stopped), S = D w of its final w
  if (checks) objective_eval<T>(L, ws, *ow, sp, tgt, D, y, ws.all, ws.all_count, false);

  FinArgs<T> fa;
  fa.W = ws.W; fa.G2 = ws.G2; fa.LB2 = ws.LB2; fa.iters = ws.iters; fa.status = ws.status; fa.err = ws.err;
  fa.w_out = w; fa.g_out = g; fa.t_out = t_out; fa.iters_out = iters_out; fa.status_out = status_out;
  fa.err_out = err_out; fa.batch = batch; fa.n = n; fa.k = k; fa.gscale_inv = T(eps_ln2);
  L.begin(KIND_OTHER);
  finalize_kernel<T><<<1184, 256, 0, L.stream>>>(fa);
  L.end();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && L.timer && L.timer->on) e = L.timer->harvest();
  return e;
}

}  // namespace otlm
