// C ABI of the OTLM solver (declared in include/otlm.h): argument validation, handle/workspace
// ownership, precision dispatch and the host-buffer variant.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/otlm.h"
#include "objective.cuh"
#include "solver.cuh"
#include "tc_solver.cuh"

using otlm::Launch;
using otlm::SolveParams;
using otlm::Workspace;

struct otlm_ctx {
  otlm_config cfg;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;        // solver workspace (one allocation)
  void* stage = nullptr;     // device staging for otlm_solve_host (allocated on first use)
  size_t stage_bytes = 0;
  int* host_flag = nullptr;  // pinned
  long long launches = 0;
  size_t elem = 4;
  otlm::Timer timer;
  bool timer_ready = false;
};

namespace {

bool valid_enum(const otlm_config& c) {
  return (c.precision == OTLM_PREC_FP32_LOG || c.precision == OTLM_PREC_FP64 || c.precision == OTLM_PREC_BF16_TC) &&
         (c.datafit >= OTLM_DATAFIT_BALANCED && c.datafit <= OTLM_DATAFIT_L2) &&
         (c.penalty >= OTLM_PENALTY_NONE && c.penalty <= OTLM_PENALTY_L2SQ);
}

size_t workspace_bytes(const otlm_config& c) {
  if (c.precision == OTLM_PREC_FP64)
    return otlm::carve_workspace<double>(nullptr, c.n_max, c.k_max, c.batch_max, nullptr);
  size_t bytes = otlm::carve_workspace<float>(nullptr, c.n_max, c.k_max, c.batch_max, nullptr);
  if (c.precision == OTLM_PREC_BF16_TC)
    bytes += otlm::carve_tc_workspace(nullptr, c.n_max, c.batch_max, nullptr) +
             otlm::carve_tc_mm(nullptr, c.n_max, c.batch_max, nullptr);
  return bytes;
}

int check_problem(const otlm_ctx* h, int batch, int n, int k, double eps, double lam, double alpha) {
  const otlm_config& c = h->cfg;
  if (batch < 1 || batch > c.batch_max || n < 2 || n > c.n_max || k < 1 || k > c.k_max) return OTLM_EINVAL;
  if (!(eps > 0) || !std::isfinite(eps)) return OTLM_EINVAL;
  if (c.datafit != OTLM_DATAFIT_BALANCED && (!(lam > 0) || !std::isfinite(lam))) return OTLM_EINVAL;
  if (!(alpha >= 0) || !std::isfinite(alpha)) return OTLM_EINVAL;
  if (c.penalty == OTLM_PENALTY_L2SQ && !(alpha > 0)) return OTLM_EINVAL;
  return OTLM_OK;
}

SolveParams params(const otlm_ctx* h, int batch, int n, int k, double eps, double lam, double alpha) {
  SolveParams sp;
  sp.batch = batch; sp.n = n; sp.k = k; sp.eps = eps; sp.lam = lam; sp.alpha = alpha;
  sp.datafit = h->cfg.datafit; sp.penalty = h->cfg.penalty; sp.max_iter = h->cfg.max_iter;
  sp.poll_every = h->cfg.poll_every; sp.tol = h->cfg.tol;
  return sp;
}

template <typename T>
int run_solve(otlm_ctx* h, const SolveParams& sp, const void* x, const void* D, const void* y, void* w, void* g,
              void* t_out, int* iters_out, void* err_out, int* status_out) {
  Workspace<T> ws;
  otlm::carve_workspace<T>(h->ws, h->cfg.n_max, h->cfg.k_max, h->cfg.batch_max, &ws);
  Launch L{h->stream, &h->launches, h->host_flag, &h->timer};
  cudaError_t e;
  if (h->cfg.precision == OTLM_PREC_BF16_TC) {
    otlm::TcWorkspace tw;
    const size_t base = otlm::carve_workspace<float>(nullptr, h->cfg.n_max, h->cfg.k_max, h->cfg.batch_max, nullptr);
    const size_t tcb = otlm::carve_tc_workspace(static_cast<char*>(h->ws) + base, h->cfg.n_max, h->cfg.batch_max, &tw);
    otlm::TcMMBuf mb;
    otlm::carve_tc_mm(static_cast<char*>(h->ws) + base + tcb, h->cfg.n_max, h->cfg.batch_max, &mb);
    e = otlm::solve_device_tc(L, reinterpret_cast<const Workspace<float>&>(ws), tw, mb, sp, (const float*)x,
                              (const float*)D, (const float*)y, (float*)w, (float*)g, (float*)t_out, iters_out,
                              (float*)err_out, status_out);
  } else {
    e = otlm::solve_device<T>(L, ws, sp, (const T*)x, (const T*)D, (const T*)y, (T*)w, (T*)g, (T*)t_out, iters_out,
                              (T*)err_out, status_out);
  }
  if (e == cudaErrorLaunchTimeout) return OTLM_ETIMEOUT;
  return e == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}

template <typename T>
int run_objective(otlm_ctx* h, const SolveParams& sp, const void* x, const void* D, const void* y, const void* w,
                  const void* g, double* primal, double* dual) {
  Workspace<T> ws;
  otlm::carve_workspace<T>(h->ws, h->cfg.n_max, h->cfg.k_max, h->cfg.batch_max, &ws);
  Launch L{h->stream, &h->launches, h->host_flag, &h->timer};
  cudaError_t e = otlm::objective_device<T>(L, ws, sp, (const T*)x, (const T*)D, (const T*)y, (const T*)w,
                                            (const T*)g, primal, dual);
  return e == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}

}  // namespace

extern "C" {

int otlm_create(otlm_handle* out, const otlm_config* cfg, void* cuda_stream) {
  if (!out) return OTLM_EINVAL;
  *out = nullptr;
  if (!cfg) return OTLM_EINVAL;
  const otlm_config& c = *cfg;
  if (c.n_max < 2 || c.k_max < 1 || c.k_max > 256 || c.batch_max < 1 || c.max_iter < 1 || c.poll_every < 1 ||
      !valid_enum(c) || !std::isfinite(c.tol))
    return OTLM_EINVAL;
  if ((size_t)c.batch_max * (size_t)c.n_max > (size_t)1 << 34) return OTLM_EINVAL;
  otlm_ctx* h = new (std::nothrow) otlm_ctx;
  if (!h) return OTLM_ENOMEM;
  h->cfg = c;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->elem = c.precision == OTLM_PREC_FP64 ? 8 : 4;
  if (cudaMalloc(&h->ws, workspace_bytes(c)) != cudaSuccess) {
    delete h;
    return OTLM_ENOMEM;
  }
  if (cudaMallocHost(&h->host_flag, sizeof(int)) != cudaSuccess) {
    cudaFree(h->ws);
    delete h;
    return OTLM_ECUDA;
  }
  *out = h;
  return OTLM_OK;
}

void otlm_destroy(otlm_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  cudaFree(h->ws);
  if (h->stage) cudaFree(h->stage);
  cudaFreeHost(h->host_flag);
  if (h->timer_ready) h->timer.destroy();
  delete h;
}

int otlm_solve(otlm_handle h, int batch, int n, int k, const void* x, const void* D, const void* y, double eps,
               double lam, double alpha, void* w, void* g, void* t_out, int* iters_out, void* err_out,
               int* status_out) {
  if (!h || !x || !D || !y || !w) return OTLM_EINVAL;
  int rc = check_problem(h, batch, n, k, eps, lam, alpha);
  if (rc != OTLM_OK) return rc;
  const SolveParams sp = params(h, batch, n, k, eps, lam, alpha);
  if (h->cfg.precision == OTLM_PREC_FP64)
    return run_solve<double>(h, sp, x, D, y, w, g, t_out, iters_out, err_out, status_out);
  return run_solve<float>(h, sp, x, D, y, w, g, t_out, iters_out, err_out, status_out);
}

int otlm_solve_host(otlm_handle h, int batch, int n, int k, const void* x, const void* D, const void* y, double eps,
                    double lam, double alpha, void* w, void* g, void* t_out, int* iters_out, void* err_out,
                    int* status_out) {
  if (!h || !x || !D || !y || !w) return OTLM_EINVAL;
  int rc = check_problem(h, batch, n, k, eps, lam, alpha);
  if (rc != OTLM_OK) return rc;
  const otlm_config& c = h->cfg;
  const size_t E = h->elem;
  const size_t bn = (size_t)c.batch_max * c.n_max, bk = (size_t)c.batch_max * c.k_max;
  // staging: x, D, y, w, g, t, err (elements), iters, status (ints)
  auto a = [](size_t v) { return otlm::align_up(v); };
  const size_t need = a(E * c.n_max) + a(E * (size_t)c.n_max * c.k_max) + 3 * a(E * bn) + a(E * bk) +
                      a(E * c.batch_max) + 2 * a(sizeof(int) * c.batch_max);
  if (!h->stage) {
    if (cudaMalloc(&h->stage, need) != cudaSuccess) return OTLM_ENOMEM;
    h->stage_bytes = need;
  }
  char* p = static_cast<char*>(h->stage);
  void* dx = p; p += a(E * c.n_max);
  void* dD = p; p += a(E * (size_t)c.n_max * c.k_max);
  void* dy = p; p += a(E * bn);
  void* dg = p; p += a(E * bn);
  void* dt = p; p += a(E * bn);
  void* dw = p; p += a(E * bk);
  void* de = p; p += a(E * c.batch_max);
  int* di = (int*)p; p += a(sizeof(int) * c.batch_max);
  int* ds = (int*)p;
  const size_t sbn = E * (size_t)batch * n, sbk = E * (size_t)batch * k;
  cudaStream_t s = h->stream;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, kind, s);
  };
  cp(dx, x, E * n, cudaMemcpyHostToDevice);
  cp(dD, D, E * (size_t)n * k, cudaMemcpyHostToDevice);
  cp(dy, y, sbn, cudaMemcpyHostToDevice);
  cp(dw, w, sbk, cudaMemcpyHostToDevice);
  if (g) cp(dg, g, sbn, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return OTLM_ECUDA;
  rc = otlm_solve(h, batch, n, k, dx, dD, dy, eps, lam, alpha, dw, g ? dg : nullptr, t_out ? dt : nullptr, di, de, ds);
  if (rc != OTLM_OK) return rc;
  cp(w, dw, sbk, cudaMemcpyDeviceToHost);
  if (g) cp(g, dg, sbn, cudaMemcpyDeviceToHost);
  if (t_out) cp(t_out, dt, sbn, cudaMemcpyDeviceToHost);
  if (iters_out) cp(iters_out, di, sizeof(int) * batch, cudaMemcpyDeviceToHost);
  if (status_out) cp(status_out, ds, sizeof(int) * batch, cudaMemcpyDeviceToHost);
  if (err_out) cp(err_out, de, E * batch, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}

int otlm_objective(otlm_handle h, int batch, int n, int k, const void* x, const void* D, const void* y, double eps,
                   double lam, double alpha, const void* w, const void* g, double* primal_out, double* dual_out) {
  if (!h || !x || !D || !y || !w || !g || !primal_out || !dual_out) return OTLM_EINVAL;
  int rc = check_problem(h, batch, n, k, eps, lam, alpha);
  if (rc != OTLM_OK) return rc;
  const SolveParams sp = params(h, batch, n, k, eps, lam, alpha);
  if (h->cfg.precision == OTLM_PREC_FP64) return run_objective<double>(h, sp, x, D, y, w, g, primal_out, dual_out);
  return run_objective<float>(h, sp, x, D, y, w, g, primal_out, dual_out);
}

long long otlm_launch_count(otlm_handle h) { return h ? h->launches : -1; }

int otlm_set_timing(otlm_handle h, int enable) {
  if (!h) return OTLM_EINVAL;
  if (enable && !h->timer_ready) {
    if (h->timer.create() != cudaSuccess) return OTLM_ECUDA;
    h->timer_ready = true;
  }
  h->timer.on = enable != 0;
  return OTLM_OK;
}

int otlm_get_timing(otlm_handle h, double* ms, long long* launches) {
  if (!h || !ms || !launches) return OTLM_EINVAL;
  if (h->timer_ready && h->timer.harvest() != cudaSuccess) return OTLM_ECUDA;
  for (int i = 0; i < otlm::KIND_COUNT; ++i) {
    ms[i] = h->timer.ms[i];
    launches[i] = h->timer.count[i];
    h->timer.ms[i] = 0.0;
    h->timer.count[i] = 0;
  }
  return OTLM_OK;
}

const char* otlm_strerror(int code) {
  switch (code) {
    case OTLM_OK: return "ok";
    case OTLM_EINVAL: return "invalid argument";
    case OTLM_ECUDA: return "CUDA runtime error";
    case OTLM_ENOMEM: return "device allocation failed";
    case OTLM_EUNSUPPORTED: return "not supported by this build";
    case OTLM_ESCRATCH: return "problem exceeds the 16 MiB static scratch of otlm_solve_noalloc";
    case OTLM_ETIMEOUT: return "a bounded device-side wait expired";
    default: return "unknown otlm status";
  }
}

}  // extern "C"
