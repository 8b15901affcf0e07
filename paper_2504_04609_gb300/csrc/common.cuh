// Device helpers shared by the OTLM kernels: precision traits, block reductions and the
// Wright omega function used by the squared-error datafit (Table 1) and the squared-l2 MM
// step (Table 2).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace otlm {

constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLog2e = 1.44269504088896340736;

// Arithmetic of one precision.  Potentials are carried in log2 units so that the hot loop feeds
// the exponent unit directly: exp2 of the FP32 path is the `ex2.approx.ftz.f32` instruction
// (one MUFU op), log2 is `lg2.approx.ftz.f32`.  The FP64 path calls CUDA's exp2/log2.
template <typename T> struct Prec;

template <> struct Prec<float> {
  static __device__ __forceinline__ float exp2(float v) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
  }
  static __device__ __forceinline__ float log2(float v) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
  }
  static __device__ __forceinline__ float rcp(float v) {  // rcp.approx.ftz.f32: within 1 ulp
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
  }
  static __device__ __forceinline__ float exp(float v) { return ::expf(v); }
  static __device__ __forceinline__ float expm1(float v) { return ::expm1f(v); }
  static __device__ __forceinline__ float log(float v) { return ::logf(v); }
  static __device__ __forceinline__ float ninf() { return -CUDART_INF_F; }
  static __device__ __forceinline__ float nan() { return CUDART_NAN_F; }
  static __device__ __forceinline__ float tiny() { return 1.17549435e-38f; }  // smallest normal
  static constexpr int kOmegaIters = 3;
  static constexpr float kUnderflowZ = -80.f;  // omega(z) = e^z to working precision below this
};

template <> struct Prec<double> {
  static __device__ __forceinline__ double exp2(double v) { return ::exp2(v); }
  static __device__ __forceinline__ double log2(double v) { return ::log2(v); }
  static __device__ __forceinline__ double exp(double v) { return ::exp(v); }
  static __device__ __forceinline__ double expm1(double v) { return ::expm1(v); }
  static __device__ __forceinline__ double log(double v) { return ::log(v); }
  static __device__ __forceinline__ double ninf() { return -CUDART_INF; }
  static __device__ __forceinline__ double nan() { return CUDART_NAN; }
  static __device__ __forceinline__ double tiny() { return 4.9406564584124654e-324; }  // smallest subnormal
  static constexpr int kOmegaIters = 5;
  static constexpr double kUnderflowZ = -700.0;
};

// Wright omega: the real solution w of w + log w = z, equal to W0(e^z) (Lambert W, principal
// branch).  Newton's method on F(w) = w + log w - z, whose step simplifies to
//   w <- w (1 + z - log w) / (1 + w)
// (the iteration underlying Lawrence, Corless & Jeffrey, ACM TOMS 38(3), 2012).  Start:
// e^z e^{-e^z} for z < -1 (w = e^{z - w}), z - log z + log z / z for z > 3 (asymptotic series),
// and 1 + (z-1)/2 + (z-1)^2/16 (Taylor expansion at z = 1, where w = 1) in between.  Five steps
// reach FP64 rounding over all finite z.  Returns 0 for z = -inf and e^z below the underflow
// threshold.  wright_omega_fast below runs the FP32 steps on the MUFU approximations.
template <typename T>
__device__ __forceinline__ T wright_omega(T z) {
  using P = Prec<T>;
  if (!(z > P::kUnderflowZ)) return (z == z) ? P::exp(z) : z;  // also maps -inf to 0
  T w;
  if (z < T(-1)) {
    T ez = P::exp(z);
    w = ez * P::exp(-ez);
  } else if (z > T(3)) {
    T lz = P::log(z);
    w = z - lz + lz / z;
  } else {
    T d = z - T(1);
    w = T(1) + d * T(0.5) + d * d * T(0.0625);
  }
#pragma unroll
  for (int it = 0; it < P::kOmegaIters; ++it) w = w * (T(1) + z - P::log(w)) / (T(1) + w);
  return w;
}

// FP32 variant for kernels that evaluate omega once per bin: the same start and three Newton
// steps, with log w = ln2 lg2(w) (lg2.approx, absolute error about 2^-22) and the division as a
// multiply by rcp.approx.  Newton corrects the errors of every step but the last, whose log error
// moves w by a relative ~1e-7 / (1 + w): FP32 rounding.  (Kernels that need omega only once per
// weight keep wright_omega<float>.)
__device__ __forceinline__ float wright_omega_fast(float z) {
  using P = Prec<float>;
  constexpr float ln2 = 0.693147180559945309f, log2e = 1.442695040888963407f;
  if (!(z > P::kUnderflowZ)) return (z == z) ? P::exp(z) : z;  // also maps -inf to 0
  float w;
  if (z < -1.f) {
    const float ez = P::exp2(z * log2e);
    w = ez * P::exp2(-ez * log2e);
  } else if (z > 3.f) {
    const float lz = P::log2(z) * ln2;
    w = z - lz + lz * P::rcp(z);
  } else {
    const float d = z - 1.f;
    w = 1.f + d * 0.5f + d * d * 0.0625f;
  }
#pragma unroll
  for (int it = 0; it < P::kOmegaIters; ++it) w = w * (1.f + z - P::log2(w) * ln2) * P::rcp(1.f + w);
  return w;
}

// Sum over a block of `nthreads` threads; `red` holds >= 32 elements of shared scratch.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) red[0] = v;
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

// Maximum over a block of `nthreads` threads; `red` holds >= 32 elements of shared scratch.
template <typename T>
__device__ __forceinline__ T block_max(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : -CUDART_INF_F;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (threadIdx.x == 0) red[0] = v;
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

}  // namespace otlm
