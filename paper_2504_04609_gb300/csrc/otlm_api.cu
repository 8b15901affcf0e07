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
#include "ragged.cuh"
#include "banded_api.h"

#include <algorithm>
#include <vector>

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
  // uneven-batch path (allocated on first use)
  int* rg_order = nullptr;         // [batch_max] queue order + 1 counter
  cudaStream_t rg_stream = nullptr;
  cudaEvent_t rg_ev[2] = {nullptr, nullptr};
  cudaGraphExec_t rg_exec = nullptr;
  unsigned char rg_key[sizeof(otlm::RaggedArgs) + 2 * sizeof(int)] = {};
  int rg_variant = 1;              // CTA size chosen by otlm_tune_ragged (default 256 threads)
  unsigned char rg_rows[otlm::RAGGED_BUCKETS] = {};  // log2 rows per thread by size bucket (0: fewest)
  long long rg_tot[3] = {0, 0, 0}; // packed sizes sum n, sum n k, sum k of the last batch
  // banded path (allocated on first use, grown when a call needs more)
  void* bd = nullptr;
  size_t bd_bytes = 0;
};

namespace {

bool valid_enum(const otlm_config& c) {
  return (c.precision == OTLM_PREC_FP32_LOG || c.precision == OTLM_PREC_FP64 || c.precision == OTLM_PREC_BF16_TC) &&
         (c.datafit >= OTLM_DATAFIT_BALANCED && c.datafit <= OTLM_DATAFIT_POISSON) &&
         (c.penalty >= OTLM_PENALTY_NONE && c.penalty <= OTLM_PENALTY_ELASTIC) &&
         (c.penalty != OTLM_PENALTY_ELASTIC || (c.beta > 0 && std::isfinite(c.beta))) &&
         c.mm_steps >= 0 && c.mm_steps <= 64 && c.check_every >= 0 && c.gap_tol >= 0 && std::isfinite(c.gap_tol) &&
         c.dw_tol >= 0 && std::isfinite(c.dw_tol) && (c.gap_tol == 0 || c.check_every > 0) &&
         (c.ragged_cta == 0 || c.ragged_cta == 128 || c.ragged_cta == 256 || c.ragged_cta == 512) &&
         std::all_of(c.ragged_rows_log2, c.ragged_rows_log2 + 16, [](int v) { return v >= 0 && v <= 5; }) &&
         c.bf16_single_until >= 0 && c.bf16_single_until < 1 &&
         (c.bf16_single_until == 0 || c.precision == OTLM_PREC_BF16_TC) &&
         (c.cost == OTLM_COST_GRID_SQ || c.cost == OTLM_COST_GRID_ABS);
}

// Byte offsets of the workspace parts: the solver state, then (tensor-core handles) the GEMM
// operands and the MM partial sums, then (check_every > 0) the objective scratch.
struct WsLayout {
  size_t base = 0, tc = 0, mm = 0, obj = 0, total = 0;
};
WsLayout ws_layout(const otlm_config& c) {
  WsLayout l;
  const bool f64 = c.precision == OTLM_PREC_FP64;
  l.base = f64 ? otlm::carve_workspace<double>(nullptr, c.n_max, c.k_max, c.batch_max, nullptr)
               : otlm::carve_workspace<float>(nullptr, c.n_max, c.k_max, c.batch_max, nullptr);
  if (c.precision == OTLM_PREC_BF16_TC) {
    l.tc = otlm::carve_tc_workspace(nullptr, c.n_max, c.k_max, c.batch_max, nullptr);
    l.mm = otlm::carve_tc_mm(nullptr, c.k_max, c.batch_max, nullptr);
  }
  if (c.check_every > 0)
    l.obj = f64 ? otlm::carve_obj_workspace<double>(nullptr, c.n_max, c.batch_max, nullptr)
                : otlm::carve_obj_workspace<float>(nullptr, c.n_max, c.batch_max, nullptr);
  l.total = l.base + l.tc + l.mm + l.obj;
  return l;
}

size_t workspace_bytes(const otlm_config& c) { return ws_layout(c).total; }

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
  sp.beta = h->cfg.beta; sp.mm_steps = h->cfg.mm_steps > 1 ? h->cfg.mm_steps : 1;
  sp.check_every = h->cfg.check_every; sp.gap_tol = h->cfg.gap_tol; sp.dw_tol = h->cfg.dw_tol;
  sp.single_until = h->cfg.bf16_single_until;
  sp.cost = h->cfg.cost == OTLM_COST_GRID_ABS ? otlm::COST_ABS : otlm::COST_SQ;
  return sp;
}

// C: dense cost [n][n] or NULL for the grid cost from x
template <typename T>
int run_solve(otlm_ctx* h, const SolveParams& sp, const void* x, const void* C, const void* D, const void* y, void* w,
              void* g, void* t_out, int* iters_out, void* err_out, int* status_out) {
  const otlm_config& c = h->cfg;
  const WsLayout lay = ws_layout(c);
  char* base = static_cast<char*>(h->ws);
  Workspace<T> ws;
  otlm::carve_workspace<T>(base, c.n_max, c.k_max, c.batch_max, &ws);
  otlm::ObjWorkspace<T> ow;
  if (lay.obj) otlm::carve_obj_workspace<T>(base + lay.base + lay.tc + lay.mm, c.n_max, c.batch_max, &ow);
  Launch L{h->stream, &h->launches, h->host_flag, &h->timer};
  cudaError_t e;
  if (c.precision == OTLM_PREC_BF16_TC) {
    otlm::TcWorkspace tw;
    otlm::carve_tc_workspace(base + lay.base, c.n_max, c.k_max, c.batch_max, &tw);
    otlm::TcMMBuf mb;
    otlm::carve_tc_mm(base + lay.base + lay.tc, c.k_max, c.batch_max, &mb);
    e = otlm::solve_device_tc(L, reinterpret_cast<const Workspace<float>&>(ws), tw, mb,
                              lay.obj ? reinterpret_cast<const otlm::ObjWorkspace<float>*>(&ow) : nullptr, sp,
                              (const float*)x, (const float*)C, (const float*)D, (const float*)y, (float*)w,
                              (float*)g, (float*)t_out, iters_out, (float*)err_out, status_out);
  } else {
    e = otlm::solve_device<T>(L, ws, lay.obj ? &ow : nullptr, sp, (const T*)x, (const T*)D, (const T*)y, (T*)w,
                              (T*)g, (T*)t_out, iters_out, (T*)err_out, status_out, (const T*)C);
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


// Validate an uneven batch on host copies of n, k, eps and the offsets, and build the
// largest-work-first order.  The packed arrays hold sum n, sum n k and sum k elements (the
// header's contract), so every problem's range must lie inside them; the kernel repeats the check
// as a backstop.
int ragged_setup(otlm_ctx* h, int batch, const int* n, const int* k, const float* eps, const long long* off_n,
                 const long long* off_D, const long long* off_k, std::vector<int>* order,
                 std::vector<int>* n_host = nullptr) {
  const otlm_config& c = h->cfg;
  if (c.precision != OTLM_PREC_FP32_LOG || c.check_every > 0 || c.dw_tol > 0 || c.cost != OTLM_COST_GRID_SQ)
    return OTLM_EUNSUPPORTED;
  if (batch < 1 || batch > c.batch_max || c.n_max > 4096) return OTLM_EINVAL;
  std::vector<int> hn(batch), hk(batch);
  std::vector<float> he(batch);
  std::vector<long long> hon(batch), hoD(batch), hok(batch);
  if (cudaMemcpy(hn.data(), n, sizeof(int) * batch, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(hk.data(), k, sizeof(int) * batch, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(he.data(), eps, sizeof(float) * batch, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(hon.data(), off_n, sizeof(long long) * batch, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(hoD.data(), off_D, sizeof(long long) * batch, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(hok.data(), off_k, sizeof(long long) * batch, cudaMemcpyDeviceToHost) != cudaSuccess)
    return OTLM_ECUDA;
  for (int p = 0; p < batch; ++p)
    if (hn[p] < 2 || hn[p] > c.n_max || hk[p] < 1 || hk[p] > c.k_max || !(he[p] > 0.f) || !std::isfinite(he[p]))
      return OTLM_EINVAL;
  long long tn = 0, tD = 0, tk = 0;
  for (int p = 0; p < batch; ++p) {
    tn += hn[p];
    tD += (long long)hn[p] * hk[p];
    tk += hk[p];
  }
  for (int p = 0; p < batch; ++p)
    if (hon[p] < 0 || hon[p] > tn - hn[p] || hoD[p] < 0 || hoD[p] > tD - (long long)hn[p] * hk[p] || hok[p] < 0 ||
        hok[p] > tk - hk[p])
      return OTLM_EINVAL;
  h->rg_tot[0] = tn; h->rg_tot[1] = tD; h->rg_tot[2] = tk;
  if (n_host) *n_host = hn;
  order->resize(batch);
  for (int p = 0; p < batch; ++p) (*order)[p] = p;
  std::stable_sort(order->begin(), order->end(),
                   [&](int a, int b) { return (long long)hn[a] * hn[a] > (long long)hn[b] * hn[b]; });
  if (!h->rg_order) {
    if (cudaMalloc(&h->rg_order, sizeof(int) * (c.batch_max + 64)) != cudaSuccess) return OTLM_ENOMEM;
    if (cudaStreamCreateWithFlags(&h->rg_stream, cudaStreamNonBlocking) != cudaSuccess) return OTLM_ECUDA;
    for (cudaEvent_t& e : h->rg_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return OTLM_ECUDA;
  }
  return OTLM_OK;
}

// Launch the persistent kernel as a captured CUDA graph on the internal stream, ordered after
// the handle's stream and before its later work.  The graph is re-instantiated only when the
// arguments or the variant change.
int ragged_run(otlm_ctx* h, const otlm::RaggedArgs& a0, int variant, bool use_graph) {
  int bps = 0;
  size_t smem = 0;
  if (otlm::ragged_prepare(variant, h->cfg.n_max, h->cfg.k_max, &bps, &smem) != cudaSuccess || bps < 1)
    return OTLM_ECUDA;
  otlm::RaggedArgs a;
  std::memcpy(&a, &a0, sizeof(a));  // padding included: the struct's bytes key the cached graph
  a.smem_floats = (int)(smem / 4);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const dim3 grid(std::max(1, std::min(sms * bps, a.batch)));
  Launch L{h->stream, &h->launches, h->host_flag, &h->timer};
  cudaError_t e = cudaEventRecord(h->rg_ev[0], h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->rg_stream, h->rg_ev[0], 0);
  if (e != cudaSuccess) return OTLM_ECUDA;
  L.begin(otlm::KIND_APPLY);
  if (use_graph) {
    unsigned char key[sizeof(h->rg_key)];
    std::memcpy(key, &a, sizeof(a));
    std::memcpy(key + sizeof(a), &variant, sizeof(int));
    const int gx = (int)grid.x;
    std::memcpy(key + sizeof(a) + sizeof(int), &gx, sizeof(int));
    if (!h->rg_exec || std::memcmp(key, h->rg_key, sizeof(key)) != 0) {
      if (h->rg_exec) {
        cudaGraphExecDestroy(h->rg_exec);
        h->rg_exec = nullptr;
      }
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(h->rg_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaMemsetAsync(a.next, 0, sizeof(int), h->rg_stream);
        otlm::ragged_launch(variant, grid, smem, h->rg_stream, a);
        e = cudaStreamEndCapture(h->rg_stream, &graph);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&h->rg_exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) return OTLM_ECUDA;
      std::memcpy(h->rg_key, key, sizeof(key));
    }
    e = cudaGraphLaunch(h->rg_exec, h->rg_stream);
  } else {
    e = cudaMemsetAsync(a.next, 0, sizeof(int), h->rg_stream);
    if (e == cudaSuccess) {
      otlm::ragged_launch(variant, grid, smem, h->rg_stream, a);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->rg_ev[1], h->rg_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->rg_ev[1], 0);
  L.end();
  return e == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}

void ragged_args(otlm_ctx* h, int batch, const int* n, const int* k, const float* eps, const long long* off_n,
                 const long long* off_D, const long long* off_k, const float* x, const float* D, const float* y,
                 double lam, double alpha, float* w, float* g, float* t_out, int* iters_out, float* err_out,
                 int* status_out, otlm::RaggedArgs* out) {
  otlm::RaggedArgs& a = *out;
  std::memset(&a, 0, sizeof(a));
  a.batch = batch; a.order = h->rg_order; a.next = h->rg_order + h->cfg.batch_max;
  a.n = n; a.k = k; a.eps = eps; a.off_n = off_n; a.off_D = off_D; a.off_k = off_k;
  a.x = x; a.D = D; a.y = y; a.w = w; a.g_in = g; a.g_out = g; a.t_out = t_out;
  a.iters = iters_out; a.err = err_out; a.status = status_out;
  a.datafit = h->cfg.datafit; a.penalty = h->cfg.penalty; a.max_iter = h->cfg.max_iter;
  a.lam = (float)lam; a.alpha = (float)alpha; a.tol = (float)h->cfg.tol;
  a.beta = (float)h->cfg.beta; a.mm_steps = h->cfg.mm_steps > 1 ? h->cfg.mm_steps : 1;
  a.n_max = h->cfg.n_max; a.k_max = h->cfg.k_max;
  a.tot_n = h->rg_tot[0]; a.tot_D = h->rg_tot[1]; a.tot_k = h->rg_tot[2];
  std::memcpy(a.rows_log2, h->rg_rows, sizeof(a.rows_log2));
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
  h->rg_variant = c.ragged_cta == 128 ? 0 : (c.ragged_cta == 512 ? 2 : 1);
  for (int b = 0; b < otlm::RAGGED_BUCKETS; ++b) h->rg_rows[b] = (unsigned char)c.ragged_rows_log2[b];
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
  if (h->rg_exec) cudaGraphExecDestroy(h->rg_exec);
  if (h->rg_order) cudaFree(h->rg_order);
  if (h->rg_stream) cudaStreamDestroy(h->rg_stream);
  if (h->bd) cudaFree(h->bd);
  for (cudaEvent_t e : h->rg_ev)
    if (e) cudaEventDestroy(e);
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
    return run_solve<double>(h, sp, x, nullptr, D, y, w, g, t_out, iters_out, err_out, status_out);
  return run_solve<float>(h, sp, x, nullptr, D, y, w, g, t_out, iters_out, err_out, status_out);
}

int otlm_solve_cost(otlm_handle h, int batch, int n, int k, const void* C, const void* D, const void* y,
                    double eps, double lam, double alpha, void* w, void* g, void* t_out, int* iters_out,
                    void* err_out, int* status_out) {
  if (!h || !C || !D || !y || !w) return OTLM_EINVAL;
  int rc = check_problem(h, batch, n, k, eps, lam, alpha);
  if (rc != OTLM_OK) return rc;
  const SolveParams sp = params(h, batch, n, k, eps, lam, alpha);
  if (h->cfg.precision == OTLM_PREC_FP64)
    return run_solve<double>(h, sp, nullptr, C, D, y, w, g, t_out, iters_out, err_out, status_out);
  return run_solve<float>(h, sp, nullptr, C, D, y, w, g, t_out, iters_out, err_out, status_out);
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

int otlm_solve_banded(otlm_handle h, int batch, int n, int hw, const float* Cd, int k, int nnz, const int* col_ptr,
                      const int* row_idx, const float* val, const float* y, double eps, double lam, double alpha,
                      float* w, float* g, float* t_out, int* iters_out, float* err_out, int* status_out) {
  if (!h || !Cd || !col_ptr || !row_idx || !val || !y || !w) return OTLM_EINVAL;
  if (h->cfg.precision != OTLM_PREC_FP32_LOG || h->cfg.mm_steps > 1 || h->cfg.check_every > 0 || h->cfg.dw_tol > 0)
    return OTLM_EUNSUPPORTED;
  if (batch < 1 || batch > h->cfg.batch_max || n < 2 || k < 1 || nnz < 1 || hw < 0 || hw > otlm::BAND_HMAX ||
      hw >= n || (long long)batch * n > (1LL << 40))
    return OTLM_EINVAL;
  if (!(eps > 0) || !std::isfinite(eps)) return OTLM_EINVAL;
  if (h->cfg.datafit != OTLM_DATAFIT_BALANCED && (!(lam > 0) || !std::isfinite(lam))) return OTLM_EINVAL;
  if (!(alpha >= 0) || !std::isfinite(alpha) || (h->cfg.penalty == OTLM_PENALTY_L2SQ && !(alpha > 0)))
    return OTLM_EINVAL;
  const size_t need = otlm::band_workspace_bytes(batch, n, k, hw, nnz);
  if (need > h->bd_bytes) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return OTLM_ECUDA;
    if (h->bd) cudaFree(h->bd);
    h->bd = nullptr;
    h->bd_bytes = 0;
    if (cudaMalloc(&h->bd, need) != cudaSuccess) {
      h->bd = nullptr;
      return OTLM_ENOMEM;
    }
    h->bd_bytes = need;
  }
  const otlm::SolveParams sp = params(h, batch, n, k, eps, lam, alpha);
  otlm::BandCall c{batch, n, k, hw, nnz, Cd, col_ptr, row_idx, val, y, w, g, t_out, iters_out, err_out, status_out};
  Launch L{h->stream, &h->launches, h->host_flag, &h->timer};
  bool invalid = false;
  const cudaError_t e = otlm::band_solve(L, h->bd, sp, c, &invalid);
  if (e != cudaSuccess) return OTLM_ECUDA;
  return invalid ? OTLM_EINVAL : OTLM_OK;
}

int otlm_solve_ragged(otlm_handle h, int batch, const int* n, const int* k, const float* eps,
                      const long long* off_n, const long long* off_D, const long long* off_k, const float* x,
                      const float* D, const float* y, double lam, double alpha, float* w, float* g, float* t_out,
                      int* iters_out, float* err_out, int* status_out) {
  if (!h || !n || !k || !eps || !off_n || !off_D || !off_k || !x || !D || !y || !w || !iters_out || !err_out ||
      !status_out)
    return OTLM_EINVAL;
  if ((h->cfg.datafit != OTLM_DATAFIT_BALANCED && !(lam > 0)) || !(alpha >= 0) ||
      (h->cfg.penalty == OTLM_PENALTY_L2SQ && !(alpha > 0)))
    return OTLM_EINVAL;
  std::vector<int> order;
  int rc = ragged_setup(h, batch, n, k, eps, off_n, off_D, off_k, &order);
  if (rc != OTLM_OK) return rc;
  if (cudaMemcpyAsync(h->rg_order, order.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, h->stream) !=
      cudaSuccess)
    return OTLM_ECUDA;
  otlm::RaggedArgs a;
  ragged_args(h, batch, n, k, eps, off_n, off_D, off_k, x, D, y, lam, alpha, w, g, t_out, iters_out, err_out,
              status_out, &a);
  rc = ragged_run(h, a, h->rg_variant, true);
  if (rc == OTLM_OK && h->timer.on && cudaStreamSynchronize(h->stream) == cudaSuccess) h->timer.harvest();
  return rc;
}

int otlm_tune_ragged(otlm_handle h, int batch, const int* n, const int* k, const float* eps,
                     const long long* off_n, const long long* off_D, const long long* off_k, const float* x,
                     const float* D, const float* y, double lam, double alpha, const float* w, int sample_every,
                     int iters, int* cta_threads_out, int* rows_log2_out) {
  if (!h || !n || !k || !eps || !off_n || !off_D || !off_k || !x || !D || !y || !w || sample_every < 1 || iters < 1)
    return OTLM_EINVAL;
  std::vector<int> order, hn;
  int rc = ragged_setup(h, batch, n, k, eps, off_n, off_D, off_k, &order, &hn);
  if (rc != OTLM_OK) return rc;
  // sample: every sample_every-th problem of the work order (so the sample spans the sizes),
  // grouped by size bucket
  std::vector<std::vector<int>> by_bucket(otlm::RAGGED_BUCKETS);
  for (int i = 0; i < batch; i += sample_every) by_bucket[otlm::ragged_bucket(hn[order[i]])].push_back(order[i]);
  // the weights' packed length sum k (the setup checked every problem's range against it)
  const size_t wn = (size_t)h->rg_tot[2];
  float *wtmp = nullptr, *etmp = nullptr;
  int *itmp = nullptr, *stmp = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaMalloc(&wtmp, sizeof(float) * wn) == cudaSuccess &&
            cudaMalloc(&etmp, sizeof(float) * batch) == cudaSuccess &&
            cudaMalloc(&itmp, sizeof(int) * batch) == cudaSuccess &&
            cudaMalloc(&stmp, sizeof(int) * batch) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
            cudaEventCreate(&e1) == cudaSuccess;
  int sms = 0, dev = 0;
  ok = ok && cudaGetDevice(&dev) == cudaSuccess &&
       cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
  const int saved_iter = h->cfg.max_iter;
  const double saved_tol = h->cfg.tol;
  unsigned char saved_rows[otlm::RAGGED_BUCKETS];
  std::memcpy(saved_rows, h->rg_rows, sizeof(saved_rows));
  h->cfg.max_iter = iters;
  h->cfg.tol = 0.0;
  // Time one bucket with one table: the bucket's sampled problems repeated to fill two waves of
  // CTAs (a throughput measure, as in the full launch; the repeats write the tuner's own buffers).
  auto time_bucket = [&](int v, const std::vector<int>& probs, float* ms_out) -> bool {
    int bps = 0;
    size_t smem = 0;
    if (otlm::ragged_prepare(v, h->cfg.n_max, h->cfg.k_max, &bps, &smem) != cudaSuccess || bps < 1) return false;
    const int len = std::min(h->cfg.batch_max, std::max((int)probs.size(), 2 * sms * bps));
    std::vector<int> list(len);
    for (int i = 0; i < len; ++i) list[i] = probs[i % probs.size()];
    otlm::RaggedArgs a;
    ragged_args(h, len, n, k, eps, off_n, off_D, off_k, x, D, y, lam, alpha, wtmp, nullptr, nullptr, itmp, etmp,
                stmp, &a);
    bool good = true;
    for (int rep = 0; good && rep < 2; ++rep) {  // the first run warms up
      good = cudaMemcpyAsync(h->rg_order, list.data(), sizeof(int) * len, cudaMemcpyHostToDevice, h->stream) ==
                 cudaSuccess &&
             cudaMemcpyAsync(wtmp, w, sizeof(float) * wn, cudaMemcpyDeviceToDevice, h->stream) == cudaSuccess &&
             cudaEventRecord(e0, h->stream) == cudaSuccess && ragged_run(h, a, v, false) == OTLM_OK &&
             cudaEventRecord(e1, h->stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
    }
    return good && cudaEventElapsedTime(ms_out, e0, e1) == cudaSuccess;
  };
  float best_total = 1e30f;
  int best_v = h->rg_variant;
  unsigned char best_rows[otlm::RAGGED_BUCKETS] = {};
  for (int v = 0; ok && v < otlm::RAGGED_VARIANTS; ++v) {
    const int nt = otlm::ragged_nt(v), rmax_l = otlm::ragged_rmax_log2(v);
    unsigned char rows[otlm::RAGGED_BUCKETS] = {};
    float total = 0.f;
    for (int b = 0; ok && b < otlm::RAGGED_BUCKETS; ++b) {
      if (by_bucket[b].empty()) continue;
      int nmax = 0;
      for (int p : by_bucket[b]) nmax = std::max(nmax, hn[p]);
      int need_l = 1;  // the fewest rows per thread that cover every sampled size (at least 2)
      while ((1 << need_l) * nt < nmax) ++need_l;
      float best_b = 1e30f;
      int best_l = need_l;
      for (int l = need_l; ok && l <= std::min(need_l + 2, rmax_l); ++l) {
        std::memcpy(h->rg_rows, rows, sizeof(rows));
        h->rg_rows[b] = (unsigned char)l;
        float ms = 0.f;
        ok = time_bucket(v, by_bucket[b], &ms);
        if (ok && ms < best_b) {
          best_b = ms;
          best_l = l;
        }
      }
      rows[b] = (unsigned char)best_l;
      total += best_b;
    }
    if (ok && total < best_total) {
      best_total = total;
      best_v = v;
      std::memcpy(best_rows, rows, sizeof(rows));
    }
  }
  h->cfg.max_iter = saved_iter;
  h->cfg.tol = saved_tol;
  cudaFree(wtmp); cudaFree(etmp); cudaFree(itmp); cudaFree(stmp);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (!ok) {
    std::memcpy(h->rg_rows, saved_rows, sizeof(saved_rows));
    return OTLM_ECUDA;
  }
  h->rg_variant = best_v;
  std::memcpy(h->rg_rows, best_rows, sizeof(best_rows));
  if (h->rg_exec) {  // the cached graph was built for the previous order buffer contents / variant
    cudaGraphExecDestroy(h->rg_exec);
    h->rg_exec = nullptr;
  }
  if (cta_threads_out) *cta_threads_out = otlm::ragged_nt(best_v);
  if (rows_log2_out)
    for (int b = 0; b < otlm::RAGGED_BUCKETS; ++b) rows_log2_out[b] = best_rows[b];
  return OTLM_OK;
}

int otlm_initial_weights(otlm_handle h, int batch, int n, int k, const void* D, const void* y, void* w_out) {
  if (!h || !D || !y || !w_out) return OTLM_EINVAL;
  const otlm_config& c = h->cfg;
  if (batch < 1 || batch > c.batch_max || n < 2 || n > c.n_max || k < 1 || k > c.k_max) return OTLM_EINVAL;
  Launch L{h->stream, &h->launches, h->host_flag, &h->timer};
  L.begin(otlm::KIND_OTHER);
  if (c.precision == OTLM_PREC_FP64) {
    Workspace<double> ws;
    otlm::carve_workspace<double>(h->ws, c.n_max, c.k_max, c.batch_max, &ws);
    otlm::cold_colsum_kernel<double><<<(k + 127) / 128, 128, 0, h->stream>>>((const double*)D, n, k, ws.xcol);
    otlm::cold_weights_kernel<double><<<batch, 256, 0, h->stream>>>((const double*)y, ws.xcol, n, k, (double*)w_out);
  } else {
    Workspace<float> ws;
    otlm::carve_workspace<float>(h->ws, c.n_max, c.k_max, c.batch_max, &ws);
    otlm::cold_colsum_kernel<float><<<(k + 127) / 128, 128, 0, h->stream>>>((const float*)D, n, k, ws.xcol);
    otlm::cold_weights_kernel<float><<<batch, 256, 0, h->stream>>>((const float*)y, ws.xcol, n, k, (float*)w_out);
  }
  L.end();
  h->launches += 1;  // two kernels, one timed region
  return cudaGetLastError() == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}

int otlm_solve_stats(otlm_handle h, int batch, void* dw_out, double* primal_out, double* dual_out) {
  if (!h || batch < 1 || batch > h->cfg.batch_max) return OTLM_EINVAL;
  const otlm_config& c = h->cfg;
  if ((primal_out || dual_out) && c.check_every < 1) return OTLM_EINVAL;
  const WsLayout lay = ws_layout(c);
  char* base = static_cast<char*>(h->ws);
  cudaError_t e = cudaSuccess;
  if (c.precision == OTLM_PREC_FP64) {
    Workspace<double> ws;
    otlm::carve_workspace<double>(base, c.n_max, c.k_max, c.batch_max, &ws);
    if (dw_out) e = cudaMemcpyAsync(dw_out, ws.dw, sizeof(double) * batch, cudaMemcpyDeviceToDevice, h->stream);
  } else {
    Workspace<float> ws;
    otlm::carve_workspace<float>(base, c.n_max, c.k_max, c.batch_max, &ws);
    if (dw_out) e = cudaMemcpyAsync(dw_out, ws.dw, sizeof(float) * batch, cudaMemcpyDeviceToDevice, h->stream);
  }
  if (lay.obj && (primal_out || dual_out)) {
    double *pr = nullptr, *du = nullptr;
    if (c.precision == OTLM_PREC_FP64) {
      otlm::ObjWorkspace<double> ow;
      otlm::carve_obj_workspace<double>(base + lay.base + lay.tc + lay.mm, c.n_max, c.batch_max, &ow);
      pr = ow.primal; du = ow.dual;
    } else {
      otlm::ObjWorkspace<float> ow;
      otlm::carve_obj_workspace<float>(base + lay.base + lay.tc + lay.mm, c.n_max, c.batch_max, &ow);
      pr = ow.primal; du = ow.dual;
    }
    if (e == cudaSuccess && primal_out)
      e = cudaMemcpyAsync(primal_out, pr, sizeof(double) * batch, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && dual_out)
      e = cudaMemcpyAsync(dual_out, du, sizeof(double) * batch, cudaMemcpyDeviceToDevice, h->stream);
  }
  return e == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
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

int otlm_check_wait_expiry(int two_sm, int* code_out) {
  if (!code_out) return OTLM_EINVAL;
  *code_out = 0;
  constexpr int M = 256, N = 256, Kd = 256;
  const size_t op = sizeof(__nv_bfloat16) * (size_t)M * Kd, outb = sizeof(float) * (size_t)M * N;
  char* buf = nullptr;
  if (cudaMalloc(&buf, 4 * op + outb + 256) != cudaSuccess) return OTLM_ENOMEM;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 4 * op + outb + 256, st);
  const __nv_bfloat16* a_hi = reinterpret_cast<const __nv_bfloat16*>(buf);
  const __nv_bfloat16* a_lo = reinterpret_cast<const __nv_bfloat16*>(buf + op);
  const __nv_bfloat16* b_hi = reinterpret_cast<const __nv_bfloat16*>(buf + 2 * op);
  const __nv_bfloat16* b_lo = reinterpret_cast<const __nv_bfloat16*>(buf + 3 * op);
  int* err = reinterpret_cast<int*>(buf + 4 * op + outb);
  otlm::tc::GemmArgs g{};
  g.out = reinterpret_cast<float*>(buf + 4 * op);
  g.M = M; g.N = N; g.Kd = Kd; g.ld_out = M; g.err = err; g.splits = 1;
  g.wait_ns = 20000000ull;  // 20 ms
  g.withhold = 1;
  if (e == cudaSuccess)
    e = two_sm ? otlm::tc::launch_gemm3_pair<otlm::tc::KIND_BF16>(a_hi, a_lo, Kd, b_hi, b_lo, Kd, M, N, Kd, g, st)
               : otlm::tc::launch_gemm3<otlm::tc::KIND_BF16>(a_hi, a_lo, Kd, b_hi, b_lo, Kd, M, N, Kd, g, st);
  int code = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&code, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (st) cudaStreamDestroy(st);
  cudaFree(buf);
  if (e != cudaSuccess) return OTLM_ECUDA;
  *code_out = code;
  return code ? OTLM_ETIMEOUT : OTLM_OK;
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
