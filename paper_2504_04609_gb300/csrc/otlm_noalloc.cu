// otlm_solve_noalloc: the FP32 batched solve with its workspace in a fixed, statically allocated
// device array instead of memory from cudaMalloc.
//
// Who needs this: callers that must not allocate device memory themselves, e.g. code running
// inside a host framework whose caching allocator owns the GPU's memory budget (a stray
// cudaMalloc there can fail under the framework's quota or fragment its pool), or latency-critical
// loops where cudaMalloc/cudaFree would synchronise the device.  Such a caller passes its inputs
// and outputs; all scratch comes from `g_scratch` below.
//
// The array is a file-scope __device__ variable: every GPU that loads this library reserves its
// kScratchBytes until the process exits, and every call on a device shares that one array, which
// keeps whatever the previous call left in it.  Calls whose work overlaps on the GPU (two
// streams, two host threads) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/otlm.h"
#include "solver.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  In host code `g_scratch` names a host-side
// stand-in, not device memory, so the address is looked up once per device with that device
// current and cached; this first lookup is the entry point's set-up.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int otlm_solve_noalloc(int batch, int n, int k, const float* x, const float* D, const float* y,
                                  double eps, double lam, double alpha, int datafit, int penalty, int max_iter,
                                  double tol, float* w, float* g, float* t_out, int* iters_out, float* err_out,
                                  int* status_out, void* cuda_stream) {
  if (!x || !D || !y || !w) return OTLM_EINVAL;
  if (batch < 1 || n < 2 || k < 1 || k > 256 || max_iter < 1) return OTLM_EINVAL;
  if (datafit < OTLM_DATAFIT_BALANCED || datafit > OTLM_DATAFIT_POISSON) return OTLM_EINVAL;
  if (penalty < OTLM_PENALTY_NONE || penalty > OTLM_PENALTY_L2SQ) return OTLM_EINVAL;
  if (!(eps > 0) || !std::isfinite(eps) || !(alpha >= 0) || !std::isfinite(alpha) || !std::isfinite(tol))
    return OTLM_EINVAL;
  if (datafit != OTLM_DATAFIT_BALANCED && (!(lam > 0) || !std::isfinite(lam))) return OTLM_EINVAL;
  if (penalty == OTLM_PENALTY_L2SQ && !(alpha > 0)) return OTLM_EINVAL;
  // the workspace this problem needs, laid out exactly as a handle's workspace
  if ((size_t)batch * (size_t)n > kScratchBytes) return OTLM_ESCRATCH;
  const size_t need = otlm::carve_workspace<float>(nullptr, n, k, batch, nullptr);
  if (need > kScratchBytes) return OTLM_ESCRATCH;

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return OTLM_ECUDA;
  otlm::Workspace<float> ws;
  otlm::carve_workspace<float>(base, n, k, batch, &ws);

  long long launches = 0;
  int poll_flag = 0;  // pageable host int: the convergence polls copy into it synchronously
  otlm::Launch L{static_cast<cudaStream_t>(cuda_stream), &launches, &poll_flag, nullptr};
  otlm::SolveParams sp;
  sp.batch = batch; sp.n = n; sp.k = k; sp.eps = eps; sp.lam = lam; sp.alpha = alpha;
  sp.datafit = datafit; sp.penalty = penalty; sp.max_iter = max_iter; sp.poll_every = 8; sp.tol = tol;
  const cudaError_t e =
      otlm::solve_device<float>(L, ws, nullptr, sp, x, D, y, w, g, t_out, iters_out, err_out, status_out);
  return e == cudaSuccess ? OTLM_OK : OTLM_ECUDA;
}
