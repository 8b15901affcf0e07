// The banded-cost, sparse-dictionary path of Algorithm 1 (kernels in banded.cuh), compiled as its
// own translation unit; otlm_api.cu reaches it through banded_api.h.
#include "banded.cuh"

namespace otlm {

size_t band_workspace_bytes(int batch, int n, int k, int h, int nnz) {
  return carve_band_workspace(nullptr, batch, n, k, h, nnz, nullptr);
}

cudaError_t band_solve(const Launch& L, void* ws, const SolveParams& sp, const BandCall& c, bool* invalid) {
  BandWorkspace bw;
  carve_band_workspace(ws, c.batch, c.n, c.k, c.h, c.nnz, &bw);
  return solve_device_band(L, bw, sp, c, invalid);
}

}  // namespace otlm
