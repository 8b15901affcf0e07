// Internal interface of the banded path between the C-ABI file and the translation unit that holds
// its kernels (otlm_banded.cu): the call's arguments, the workspace size and the solve.
#pragma once

#include "solver.cuh"

namespace otlm {

constexpr int BAND_HMAX = 64;  // largest half-width of the cost band

// One banded solve: inputs as otlm_solve_banded (device pointers).
struct BandCall {
  int batch, n, k, h, nnz;
  const float* Cd;
  const int* col_ptr;
  const int* row_idx;
  const float* val;
  const float* y;
  float* w;
  float* g;
  float* t_out;
  int* iters_out;
  float* err_out;
  int* status_out;
};

// Bytes of device workspace for a banded solve of this shape.
size_t band_workspace_bytes(int batch, int n, int k, int h, int nnz);

// Runs the solve on `ws` (band_workspace_bytes bytes).  Returns the first CUDA error; *invalid is
// set when the band or the dictionary is malformed (checked on the device before use).
cudaError_t band_solve(const Launch& L, void* ws, const SolveParams& sp, const BandCall& c, bool* invalid);

}  // namespace otlm
