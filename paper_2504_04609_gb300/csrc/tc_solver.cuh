// Batched scaling iteration with the two kernel applies and both dictionary contractions on the
// tensor cores, for a batch sharing one grid and one dictionary.
//
// Linear domain with a per-problem shift: the source apply is
//   a_pi = sum_j K_ij u1_pj = 2^{M_p} sum_j K_ij V_pj,   V_pj = 2^{G2_pj - M_p},  M_p = max_j G2_pj,
// so every V lies in (0, 1] and the GEMM K V^T (tc_gemm.cuh, BF16 hi/lo) returns the raw sums;
// log2 a_pi = M_p + log2(sum).  The target apply is the same with U_pi = 2^{F2_pi - M'_p}.  K is
// symmetric for the squared distance on a grid, so one matrix serves both applies.  The MM step
// (Table 2) and the source step s = D w are GEMMs with the shared dictionary (TF32 hi/lo, ~21 bits:
// w and s must stay well inside the 1e-5 stopping tolerance).  Per iteration:
//   prep_src  : datafit step from the previous target sums (Table 1), then the source operand V
//   gemm      : source sums into ACC_src[it & 1] (BF16)
//   violation : source-marginal violation from the ratio of raw sums, stopping decision (it > 0),
//               and the MM log ratios r_i = log2(a_i / s_i) as a TF32 hi/lo operand
//   dtr gemm  : NU = D^T r per problem (TF32, reduction over bins split across CTAs)
//   wupd      : the weight update of Table 2, skipping problems that have just stopped
//   dw gemm   : s = D w per problem (TF32)
//   compact   : drop finished problems
//   operand   : F2 = log2 s - log2 a, the target shift and mass, then the target operand U
//   gemm      : target sums into ACC_tgt (BF16)
// dtr, wupd and dw run over the slots as they were before compaction, so the operands that the
// violation and wupd kernels write row by slot need no re-gathering.
// A sum below 2^-90 of the problem's shift (a row whose significant terms all lie far below the
// problem's largest term, e.g. far from the support under a KL or TV datafit; there the BF16 lo
// parts and products reach FP32's subnormal range and flush, down to a sum that underflows
// entirely) is listed by the GEMM epilogue and recomputed exactly (two-pass log-sum-exp for that
// row) by tc_fixup_kernel, which runs after each apply and spreads the listed rows over the GPU.
#pragma once

#include <cuda_bf16.h>

#include "kernels.cuh"
#include "solver.cuh"
#include "tc_gemm.cuh"

namespace otlm {

// Small batches leave the applies with fewer 128 x 128 output tiles than SMs (a single target at
// n = 8192 has 64), so for batches up to TC_SMALL_BATCH the reduction of each apply is split into up
// to TC_APPLY_SPLITS ranges whose partial sums are added by tc_split_reduce_kernel.
constexpr int TC_SMALL_BATCH = 64, TC_APPLY_SPLITS = 16;

struct TcWorkspace {
  __nv_bfloat16 *Khi, *Klo;  // [n][ld]
  __nv_bfloat16 *Kthi, *Ktlo;  // [n][ld] K^T, built only for a dense (possibly non-symmetric) cost
  __nv_bfloat16 *Vhi, *Vlo;  // [batch][ld], rows in active-slot order (source and target operands)
  float* ACC_src[2];         // [batch][n] raw source sums, ping-pong by iteration parity
  float* ACC_tgt;            // [batch][n] raw target sums
  float* Msrc[2];            // [batch] source shifts, ping-pong
  float* Mtgt;               // [batch] target shifts
  int* err;                  // GEMM error flag
  int* hilo;                 // [0] 0: the applies use the single BF16 product, 1: hi/lo (three
                             // products); [1] the value the iteration's source apply was launched with
  int2* fix_list;            // [batch x n] underflowed sums (problem, row) listed by a GEMM
  unsigned long long* fix_cnt;  // [2] list lengths: source GEMM, target GEMM
  unsigned long long fix_cap;
  float *Dhi, *Dlo;          // [n][kp] dictionary as TF32 hi/lo (A operand of s = D w)
  float *Dthi, *Dtlo;        // [k][ld] transposed dictionary as TF32 hi/lo (A operand of D^T r)
  float *Whi, *Wlo;          // [batch][kp] weights by slot (B operand of s = D w)
  float *Rhi, *Rlo;          // [batch][ld] log ratios by slot (B operand of D^T r)
  int ld;                    // row pitch of the [.][n] operands (multiple of 64 elements)
  int kp;                    // row pitch of the [.][k] operands (k_max rounded up to 4)
  float* ACCP;               // [TC_APPLY_SPLITS][min(batch_max, TC_SMALL_BATCH) x n] split partial sums
};

// A raw GEMM sum is a sum of positive terms, so it is >= 0.  A row the fix-up recomputed exactly
// is stored as the NEGATIVE offset log2(sum) - M (below -126, as the row underflowed), so one
// helper recovers log2 of the sum for every consumer: raw > 0, encoded < 0, 0 = empty sum.
__device__ __forceinline__ float tc_log2_sum(float a, float m) {
  return a > 0.f ? m + Prec<float>::log2(a) : (a < 0.f ? m + a : -CUDART_INF_F);
}

inline int tc_ld(int n) { return (n + 63) / 64 * 64; }

inline size_t carve_tc_workspace(void* base, int n_max, int k_max, int batch_max, TcWorkspace* ws) {
  const int ld = tc_ld(n_max), kp = (k_max + 3) / 4 * 4;
  size_t off = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* p = b ? b + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  TcWorkspace w;
  w.ld = ld;
  w.Khi = (__nv_bfloat16*)take(2 * (size_t)n_max * ld);
  w.Klo = (__nv_bfloat16*)take(2 * (size_t)n_max * ld);
  w.Kthi = (__nv_bfloat16*)take(2 * (size_t)n_max * ld);
  w.Ktlo = (__nv_bfloat16*)take(2 * (size_t)n_max * ld);
  w.Vhi = (__nv_bfloat16*)take(2 * (size_t)batch_max * ld);
  w.Vlo = (__nv_bfloat16*)take(2 * (size_t)batch_max * ld);
  w.ACC_src[0] = (float*)take(4 * (size_t)batch_max * n_max);
  w.ACC_src[1] = (float*)take(4 * (size_t)batch_max * n_max);
  w.ACC_tgt = (float*)take(4 * (size_t)batch_max * n_max);
  w.Msrc[0] = (float*)take(4 * (size_t)batch_max);
  w.Msrc[1] = (float*)take(4 * (size_t)batch_max);
  w.Mtgt = (float*)take(4 * (size_t)batch_max);
  w.err = (int*)take(64);
  w.hilo = (int*)take(64);
  w.fix_cap = (unsigned long long)batch_max * n_max;
  w.fix_list = (int2*)take(8 * (size_t)batch_max * n_max);
  w.fix_cnt = (unsigned long long*)take(64);
  w.ACCP = (float*)take(4 * (size_t)TC_APPLY_SPLITS * (batch_max < TC_SMALL_BATCH ? batch_max : TC_SMALL_BATCH) *
                        n_max);
  w.kp = kp;
  w.Dhi = (float*)take(4 * (size_t)n_max * kp);
  w.Dlo = (float*)take(4 * (size_t)n_max * kp);
  w.Dthi = (float*)take(4 * (size_t)k_max * ld);
  w.Dtlo = (float*)take(4 * (size_t)k_max * ld);
  w.Whi = (float*)take(4 * (size_t)batch_max * kp);
  w.Wlo = (float*)take(4 * (size_t)batch_max * kp);
  w.Rhi = (float*)take(4 * (size_t)batch_max * ld);
  w.Rlo = (float*)take(4 * (size_t)batch_max * ld);
  if (ws) *ws = w;
  return off;
}

// x = hi + lo with hi and lo rounded to TF32 (10 explicit mantissa bits each, round to nearest
// with ties away, the rounding cvt.rna.tf32.f32 provides); hi + lo carries ~21 bits of x.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void tf32_split(float x, float* hi, float* lo) {
  const float h = tf32_rna(x);
  *hi = h;
  *lo = tf32_rna(x - h);
}

// The dictionary D [n][k] as TF32 hi/lo, row-major [n][kp] and transposed [k][ld] (padding columns
// are never read: the tensor maps stop at k and n).
__global__ void tc_dsplit_kernel(const float* D, int n, int k, int kp, int ld, float* Dhi, float* Dlo, float* Dthi,
                                 float* Dtlo) {
  const size_t nk = (size_t)n * k;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nk; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), j = (int)(e - (size_t)i * k);
    float hi, lo;
    tf32_split(D[e], &hi, &lo);
    Dhi[(size_t)i * kp + j] = hi;
    Dlo[(size_t)i * kp + j] = lo;
    Dthi[(size_t)j * ld + i] = hi;
    Dtlo[(size_t)j * ld + i] = lo;
  }
}

// K = 2^{-(xt_i - xt_j)^2} (or 2^{-|xt_i - xt_j|} for the absolute-distance cost) as a BF16 hi/lo
// pair, [n][ld] (columns >= n left untouched: the tensor maps stop at column n).
__global__ void kbuild_kernel(const float* xt, int n, int ld, __nv_bfloat16* Khi, __nv_bfloat16* Klo, int abs_cost) {
  const size_t nn = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (size_t)i * n);
    const float d = xt[i] - xt[j];
    const float k = Prec<float>::exp2(abs_cost ? -fabsf(d) : -d * d);
    const __nv_bfloat16 hi = __float2bfloat16_rn(k);
    Khi[(size_t)i * ld + j] = hi;
    Klo[(size_t)i * ld + j] = __float2bfloat16_rn(k - __bfloat162float(hi));
  }
}

// Split applies: the problem's sums are the partial-sum planes added in order; sums below
// tc::EXACT_BELOW are listed for the fix-up as the GEMM epilogue lists them when the reduction is
// not split.
__global__ void tc_split_reduce_kernel(const float* part, int splits, size_t plane, const int* active,
                                       const int* n_active, int n, float* acc, int2* fix_list,
                                       unsigned long long* fix_cnt, unsigned long long fix_cap) {
  const size_t total = (size_t)(*n_active) * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int slot = (int)(e / n), i = (int)(e - (size_t)slot * n);
    const int p = active[slot];
    const size_t idx = (size_t)p * n + i;
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[z * plane + idx];
    acc[idx] = s;
    if (!(s >= tc::EXACT_BELOW)) {
      const unsigned long long f = atomicAdd(fix_cnt, 1ull);
      if (f < fix_cap) fix_list[f] = make_int2(p, i);
    }
  }
}

// K = 2^{-C_ij c} (c = 1 / (eps ln2)) and its transpose from a dense cost C [n][n] (row i = source
// bin, column j = target bin; +inf allowed: no transport), both as BF16 hi/lo [n][ld].  32 x 32
// tiles through shared memory keep the reads of C and the writes of both matrices coalesced.
__global__ void __launch_bounds__(256) kdense_kernel(const float* C, int n, int ld, float c, __nv_bfloat16* Khi,
                                                     __nv_bfloat16* Klo, __nv_bfloat16* Kthi, __nv_bfloat16* Ktlo) {
  __shared__ float tile[32][33];
  const int tiles = (n + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int t = blockIdx.x; t < tiles * tiles; t += gridDim.x) {
    const int i0 = (t / tiles) * 32, j0 = (t % tiles) * 32;
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int i = i0 + r, j = j0 + tx;
      float kv = 0.f;
      if (i < n && j < n) {
        kv = Prec<float>::exp2(-C[(size_t)i * n + j] * c);
        const __nv_bfloat16 hi = __float2bfloat16_rn(kv);
        Khi[(size_t)i * ld + j] = hi;
        Klo[(size_t)i * ld + j] = __float2bfloat16_rn(kv - __bfloat162float(hi));
      }
      tile[r][tx] = kv;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {  // row j0 + r of K^T = column j0 + r of K
      const int j = j0 + r, i = i0 + tx;
      if (i < n && j < n) {
        const float kv = tile[tx][r];
        const __nv_bfloat16 hi = __float2bfloat16_rn(kv);
        Kthi[(size_t)j * ld + i] = hi;
        Ktlo[(size_t)j * ld + i] = __float2bfloat16_rn(kv - __bfloat162float(hi));
      }
    }
  }
}

// Exact fix-up of the sums a GEMM listed as underflowed, one CTA of 256 threads per listed
// (problem p, row i) so that a row costs a few memory round trips, not n / 32:
//   L = log2 sum_j 2^(in_pj - cost_ij)     (two passes over j: max, then sum; cost in log2 units)
// stored as the negative offset L - M_p (decoded by tc_log2_sum); an empty sum stays 0.  in = G2
// and M = Msrc for the source sums, in = F2 and M = Mtgt for the target sums.  The source and
// target GEMMs count into fix_cnt[0] and fix_cnt[1]; each fix-up reads its own count and clears the
// other, which the next GEMM appends to.  With nothing listed every CTA leaves after one load.
constexpr int TC_FIX_GRID = 4 * 152;

// The exponent of term j of row i in log2 units: the grid cost (xt_i - xt_j)^2 or |xt_i - xt_j|,
// or a dense cost C c read along row i (trans = 0) or column i (trans = 1: a target sum of the
// transposed kernel).
struct TcCost {
  const float* xt;  // scaled grid, when C is NULL
  const float* C;   // dense cost [n][n] or NULL
  float c;          // 1 / (eps ln2)
  int trans;
  int abs_cost;     // grid cost |xt_i - xt_j|
  __device__ __forceinline__ float operator()(int i, int j, int n) const {
    if (!C) {
      const float d = xt[i] - xt[j];
      return abs_cost ? fabsf(d) : d * d;
    }
    return (trans ? C[(size_t)j * n + i] : C[(size_t)i * n + j]) * c;
  }
};

__global__ void __launch_bounds__(256) tc_fixup_kernel(const int2* list, const unsigned long long* cnt,
                                                       unsigned long long* cnt_next, unsigned long long cap, int n,
                                                       TcCost cost, const float* in, float* acc,
                                                       const float* mshift) {
  using P = Prec<float>;
  __shared__ float red[32];
  const unsigned long long c = *cnt < cap ? *cnt : cap;
  if (blockIdx.x == 0 && threadIdx.x == 0) *cnt_next = 0;
  for (unsigned long long e = blockIdx.x; e < c; e += gridDim.x) {
    const int2 pi = list[e];
    const float* inp = in + (size_t)pi.x * n;
    float mx = -CUDART_INF_F;
#pragma unroll 4
    for (int j = threadIdx.x; j < n; j += blockDim.x) mx = fmaxf(mx, inp[j] - cost(pi.y, j, n));
    mx = block_max(mx, red);
    float sum = 0.f;
    if (mx > -CUDART_INF_F) {
#pragma unroll 4
      for (int j = threadIdx.x; j < n; j += blockDim.x) sum += P::exp2((inp[j] - mx) - cost(pi.y, j, n));
    }
    sum = block_sum(sum, red);
    if (threadIdx.x == 0) {
      const float L = sum > 0.f ? mx + P::log2(sum) : -CUDART_INF_F;
      // a representable sum is stored raw; an underflowing one as its negative log2 offset
      const float off = L - mshift[pi.x];
      acc[(size_t)pi.x * n + pi.y] = !(L > -CUDART_INF_F) ? 0.f : (off >= -126.f ? P::exp2(off) : off);
    }
  }
}

struct TcIterArgs {
  const int* active;
  const int* n_active;
  int n, k, ld, it, max_iter, datafit, penalty;
  float tol, eps, alpha, beta, kl_coef, tv_bound, lam_over_eps, log_lam_over_eps;
  const float* y;
  const float* D;
  const float* Dt;
  const float* xcol;
  float* G2;
  float* S;
  float* F2;
  float* W;
  float* mass;
  float* err;
  float* dw;         // [P] ||dw||_1 / ||w||_1 of the last weight update
  float* Wprev;      // [P][k] weights before the last update
  const int* gap_ok; // [P] gap test of this iteration's check
  int gap_check, gap_on;
  float dw_tol;
  float single_until;  // > 0: switch the applies to hi/lo once a violation is <= this
  int* done;
  int* iters;
  int* status;
  TcWorkspace t;
};

// ---- per-problem row kernels (one CTA per active slot) -----------------------------------------
// With EPT > 0 the row lives in registers: thread t holds bins j = e * NT + t (e < EPT), so each
// load instruction of a warp is one contiguous 128-byte segment and every load of a pass is issued
// before its first use; n <= EPT * NT.  EPT = 0 streams the row through global memory (any n).
// tc_row_cfg picks the smallest register configuration that holds n.
enum { ROW_256x4 = 0, ROW_256x8 = 1, ROW_256x16 = 2, ROW_1024x16 = 3, ROW_STREAM = 4 };
inline int tc_row_cfg(int n) {
  return n <= 1024 ? ROW_256x4 : n <= 2048 ? ROW_256x8 : n <= 4096 ? ROW_256x16 : n <= 16384 ? ROW_1024x16 : ROW_STREAM;
}
#define TC_ROW_LAUNCH(KERNEL, CFG, GRID, STREAM, ...)                                       \
  do {                                                                                      \
    switch (CFG) {                                                                          \
      case ROW_256x4: KERNEL<256, 4><<<(GRID), 256, 0, (STREAM)>>>(__VA_ARGS__); break;     \
      case ROW_256x8: KERNEL<256, 8><<<(GRID), 256, 0, (STREAM)>>>(__VA_ARGS__); break;     \
      case ROW_256x16: KERNEL<256, 16><<<(GRID), 256, 0, (STREAM)>>>(__VA_ARGS__); break;   \
      case ROW_1024x16: KERNEL<1024, 16><<<(GRID), 1024, 0, (STREAM)>>>(__VA_ARGS__); break; \
      default: KERNEL<256, 0><<<(GRID), 256, 0, (STREAM)>>>(__VA_ARGS__); break;            \
    }                                                                                       \
  } while (0)

// Datafit step (Table 1) in log2 units: the new target potential from log2 of the target sum v and
// the target bin y.
__device__ __forceinline__ float tc_datafit(const TcIterArgs& A, float v, float yv) {
  using P = Prec<float>;
  switch (A.datafit) {
    case DF_BALANCED: return P::log2(yv) - v;
    case DF_KL: return A.kl_coef * (P::log2(yv) - v);
    case DF_TV: return fminf(fmaxf(P::log2(yv) - v, -A.tv_bound), A.tv_bound);
    default: {  // L2 or Poisson (reading A7; -lam where y = 0), one Wright omega
      const bool pois = A.datafit == DF_POISSON;
      if (pois && !(yv > 0.f)) return -A.tv_bound;
      const float l2c = pois ? A.log_lam_over_eps * float(kLog2e) + P::log2(yv) : 0.f;
      const float z = pois ? (l2c - v) * float(kLn2) + A.lam_over_eps
                           : A.log_lam_over_eps + v * float(kLn2) + A.lam_over_eps * yv;
      const float om = wright_omega_fast(z);
      return pois ? l2c - P::log2(om) - v : (A.lam_over_eps * yv - om) * float(kLog2e);
    }
  }
}

__device__ __forceinline__ void tc_store_operand(float v, __nv_bfloat16* hi_row, __nv_bfloat16* lo_row, int j) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  hi_row[j] = hi;
  lo_row[j] = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Datafit step from the previous target sums (it > 0), then the source operand row
// V_j = 2^{G2_j - M} with M = max_j G2_j (0 when every term vanishes).
template <int NT, int EPT>
__global__ void __launch_bounds__(NT) tc_prep_src_kernel(TcIterArgs A) {
  using P = Prec<float>;
  __shared__ float red[32];
  const int slot = blockIdx.x;
  // the product count the coming source apply takes (it reads hilo[0] at launch; nothing changes it
  // before then), for the stopping decision after it
  if (slot == 0 && threadIdx.x == 0) A.t.hilo[1] = A.t.hilo[0];
  if (slot >= *A.n_active) return;
  const int p = A.active[slot], n = A.n;
  float* G2 = A.G2 + (size_t)p * n;
  const float* acc = A.t.ACC_tgt + (size_t)p * n;
  const float* y = A.y + (size_t)p * n;
  const float mt = A.t.Mtgt[p];
  __nv_bfloat16* vhi = A.t.Vhi + (size_t)slot * A.t.ld;
  __nv_bfloat16* vlo = A.t.Vlo + (size_t)slot * A.t.ld;
  float m = -CUDART_INF_F;
  if constexpr (EPT > 0) {
    float g[EPT];
    if (A.it > 0) {
      float a[EPT], yv[EPT];
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int j = e * NT + threadIdx.x;
        a[e] = j < n ? acc[j] : 0.f;
        yv[e] = j < n ? y[j] : 0.f;
      }
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int j = e * NT + threadIdx.x;
        g[e] = tc_datafit(A, tc_log2_sum(a[e], mt), yv[e]);
        if (j < n) G2[j] = g[e];
      }
    } else {
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int j = e * NT + threadIdx.x;
        g[e] = j < n ? G2[j] : -CUDART_INF_F;
      }
    }
#pragma unroll
    for (int e = 0; e < EPT; ++e)
      if (e * NT + threadIdx.x < n) m = fmaxf(m, g[e]);
    m = block_max(m, red);
    if (!(m > -CUDART_INF_F)) m = 0.f;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int j = e * NT + threadIdx.x;
      if (j < n) tc_store_operand(P::exp2(g[e] - m), vhi, vlo, j);
    }
  } else {
    for (int j = threadIdx.x; j < n; j += NT) {
      const float g = A.it > 0 ? tc_datafit(A, tc_log2_sum(acc[j], mt), y[j]) : G2[j];
      if (A.it > 0) G2[j] = g;
      m = fmaxf(m, g);
    }
    m = block_max(m, red);
    if (!(m > -CUDART_INF_F)) m = 0.f;
    for (int j = threadIdx.x; j < n; j += NT) tc_store_operand(P::exp2(G2[j] - m), vhi, vlo, j);
  }
  if (threadIdx.x == 0) A.t.Msrc[A.it & 1][p] = m;
}

// Violation of the previous iteration's plan and the stopping decision (it > 0):
// e = sum_i S_i |a_new_i / a_old_i - 1| / sum_i S_i from the raw sums.  The shift difference of
// two nearby FP32 numbers is exact, so the ratio keeps FP32 relative precision.  Every iteration
// also writes the MM log ratios r_i = log2(a_i / s_i) (0 where s_i = 0) as the TF32 hi/lo row
// `slot` of the D^T r operand.
__device__ __forceinline__ float tc_violation_term(float s, float an, float ao, float mc, float mo, float f,
                                                   bool check, float* r) {
  using P = Prec<float>;
  *r = 0.f;
  if (!(s > 0.f)) return 0.f;
  const float la = tc_log2_sum(an, mc);
  *r = la - P::log2(s);
  if (!check) return 0.f;
  const float ratio = (an > 0.f && ao > 0.f) ? an / ao * f : P::exp2(la - tc_log2_sum(ao, mo));
  return s * fabsf(ratio - 1.f);
}

// RATIO_ONLY: the log ratios alone, without the convergence check (the MM steps after the first
// of an iteration, which reuse a = K u1)
template <int NT, int EPT, bool RATIO_ONLY>
__device__ __forceinline__ void tc_violation_body(const TcIterArgs& A) {
  using P = Prec<float>;
  __shared__ float red[32];
  const int slot = blockIdx.x;
  if (slot >= *A.n_active) return;
  const int p = A.active[slot], n = A.n, cur = A.it & 1;
  const float* acc = A.t.ACC_src[cur] + (size_t)p * n;
  const float* acc_old = A.t.ACC_src[cur ^ 1] + (size_t)p * n;
  const float* S = A.S + (size_t)p * n;
  float* rhi = A.t.Rhi + (size_t)slot * A.t.ld;
  float* rlo = A.t.Rlo + (size_t)slot * A.t.ld;
  const float mc = A.t.Msrc[cur][p], mo = A.t.Msrc[cur ^ 1][p];
  const float f = P::exp2(mc - mo);
  const bool check = !RATIO_ONLY && A.it > 0;
  float part = 0.f;
  if constexpr (EPT > 0) {
    float s[EPT], an[EPT], ao[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int j = e * NT + threadIdx.x;
      s[e] = j < n ? S[j] : 0.f;
      an[e] = j < n ? acc[j] : 0.f;
      ao[e] = (check && j < n) ? acc_old[j] : 0.f;
    }
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int j = e * NT + threadIdx.x;
      float r;
      part += tc_violation_term(s[e], an[e], ao[e], mc, mo, f, check, &r);
      if (j < n) tf32_split(r, rhi + j, rlo + j);
    }
  } else {
    for (int j = threadIdx.x; j < n; j += NT) {
      float r;
      part += tc_violation_term(S[j], acc[j], check ? acc_old[j] : 0.f, mc, mo, f, check, &r);
      tf32_split(r, rhi + j, rlo + j);
    }
  }
  if (!check) return;
  part = block_sum(part, red);
  // weight change of the previous iteration's update (k <= 256 entries)
  float num = 0.f, den = 0.f;
  for (int j = threadIdx.x; j < A.k; j += NT) {
    const float wv = A.W[(size_t)p * A.k + j];
    num += fabsf(wv - A.Wprev[(size_t)p * A.k + j]);
    den += fabsf(wv);
  }
  num = block_sum(num, red);
  den = block_sum(den, red);
  if (threadIdx.x == 0) {
    const float e = part / A.mass[p];
    const float dw = num / den;
    A.err[p] = e;
    A.dw[p] = dw;
    // the precision schedule: the first problem whose violation reaches single_until switches every
    // later apply to the hi/lo products (a violation this large is far from any stop at tol)
    if (A.single_until > 0.f && e <= A.single_until) atomicExch(A.t.hilo, 1);
    // a converged stop needs this iteration's source sums from the hi/lo products
    const bool src_hilo = !(A.single_until > 0.f) || A.t.hilo[1] != 0;
    const int st = stop_decision<float>(e, dw, A.tol, A.dw_tol, A.gap_on != 0,
                                        A.gap_check && A.gap_ok && A.gap_ok[p], A.it, A.max_iter, src_hilo);
    if (st >= 0) {
      A.status[p] = st;
      A.iters[p] = A.it;
      A.done[p] = 1;
    }
  }
}

template <int NT, int EPT>
__global__ void __launch_bounds__(NT, NT == 256 ? 4 : 1) tc_violation_kernel(TcIterArgs A) {
  tc_violation_body<NT, EPT, false>(A);
}

template <int NT, int EPT>
__global__ void __launch_bounds__(NT, NT == 256 ? 4 : 1) tc_ratio_kernel(TcIterArgs A) {
  tc_violation_body<NT, EPT, true>(A);
}

// ---- the MM step and the source step around the two TF32 dictionary GEMMs ----------------------
//
// dtr gemm : NU[z][slot][j] = sum_{i in split z} D_ij r_slot,i   (A = D^T [k][ld], B = R [slot][ld])
// wupd     : w update of Table 2 from nu = log w + (ln2 / x_j) sum_z NU[z] (splits added in order)
// dw gemm  : S[p][i] = sum_j D_ij w_pj                           (A = D [n][kp], B = W [slot][kp])
// operand  : per slot, F2, the shift max(F2) and mass sum(S), then the target operand row.
constexpr int TC_MAX_SPLITS = 16;

struct TcMMBuf {
  float* NU;      // [TC_MAX_SPLITS][batch_max][ldnu] partial sums of D^T r
  int ldnu;       // k_max rounded up to 4
  size_t plane;   // batch_max * ldnu: elements per split
};

inline size_t carve_tc_mm(void* base, int k_max, int batch_max, TcMMBuf* mb) {
  size_t off = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* p = b ? b + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  TcMMBuf m;
  m.ldnu = (k_max + 3) / 4 * 4;
  m.plane = (size_t)batch_max * m.ldnu;  // rows of a split are written with pitch ldnu
  m.NU = (float*)take(4 * (size_t)TC_MAX_SPLITS * m.plane);
  if (mb) *mb = m;
  return off;
}

// One thread per (slot, j) of the slots before compaction.  A problem that has just stopped keeps
// its weights (and with update = 0 every problem does); every slot writes its weight row as the
// TF32 hi/lo B operand of s = D w.
// save_prev: the first update of an iteration also keeps the weights it starts from (Wprev), for
// the weight-change measure of the next stopping decision.
__global__ void __launch_bounds__(256) tc_wupd_kernel(TcIterArgs A, TcMMBuf M, int splits, int update,
                                                      int save_prev) {
  using P = Prec<float>;
  const int na = *A.n_active, k = A.k;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int slot = e / k, j = e - slot * k;
  if (slot >= na) return;
  const int p = A.active[slot];
  float wn = A.W[(size_t)p * k + j];
  if (update && !A.done[p]) {
    if (save_prev) A.Wprev[(size_t)p * k + j] = wn;
    float sum = 0.f;
    for (int z = 0; z < splits; ++z) sum += M.NU[z * M.plane + (size_t)slot * M.ldnu + j];
    const float xj = A.xcol[j];
    const float nu = P::log(wn) + sum * float(kLn2) / xj;
    const float shift = (A.penalty == PEN_L1 || A.penalty == PEN_ELASTIC) ? A.alpha / (A.eps * xj) : 0.f;
    if (A.penalty == PEN_L2SQ || A.penalty == PEN_ELASTIC) {
      const float c = (A.penalty == PEN_ELASTIC ? A.beta : A.alpha) / (A.eps * xj);
      wn = wright_omega_fast(P::log(c) + nu - shift) / c;
    } else wn = P::exp(nu - shift);
    A.W[(size_t)p * k + j] = wn;
  }
  tf32_split(wn, A.t.Whi + (size_t)slot * A.t.kp + j, A.t.Wlo + (size_t)slot * A.t.kp + j);
}

// One CTA per active slot (after compaction): F2_i = log2 S_i - log2 a_i (-inf where S_i = 0), the
// target shift M' = max_i F2_i, the mass sum_i S_i, then U_i = 2^{F2_i - M'} as BF16 hi/lo.
template <int NT, int EPT>
__global__ void __launch_bounds__(NT) tc_operand_kernel(TcIterArgs A) {
  using P = Prec<float>;
  __shared__ float red[32];
  const int slot = blockIdx.x;
  if (slot >= *A.n_active) return;
  const int p = A.active[slot], n = A.n, cur = A.it & 1;
  const float* S = A.S + (size_t)p * n;
  const float* acc = A.t.ACC_src[cur] + (size_t)p * n;
  float* F2 = A.F2 + (size_t)p * n;
  __nv_bfloat16* vhi = A.t.Vhi + (size_t)slot * A.t.ld;
  __nv_bfloat16* vlo = A.t.Vlo + (size_t)slot * A.t.ld;
  const float mc = A.t.Msrc[cur][p];
  float fm = -CUDART_INF_F, ms = 0.f;
  if constexpr (EPT > 0) {
    float f2[EPT];
    {
      float sv[EPT], av[EPT];
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int j = e * NT + threadIdx.x;
        sv[e] = j < n ? S[j] : 0.f;
        av[e] = j < n ? acc[j] : 0.f;
      }
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int j = e * NT + threadIdx.x;
        f2[e] = sv[e] > 0.f ? P::log2(sv[e]) - tc_log2_sum(av[e], mc) : P::ninf();
        if (j < n) F2[j] = f2[e];
        fm = fmaxf(fm, f2[e]);
        ms += sv[e];
      }
    }
    fm = block_max(fm, red);
    ms = block_sum(ms, red);
    const float m = fm > -CUDART_INF_F ? fm : 0.f;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int j = e * NT + threadIdx.x;
      if (j < n) tc_store_operand(P::exp2(f2[e] - m), vhi, vlo, j);
    }
    if (threadIdx.x == 0) {
      A.mass[p] = ms;
      A.t.Mtgt[p] = m;
    }
  } else {
    for (int i = threadIdx.x; i < n; i += NT) {
      const float s = S[i];
      const float f2 = s > 0.f ? P::log2(s) - tc_log2_sum(acc[i], mc) : P::ninf();
      F2[i] = f2;
      fm = fmaxf(fm, f2);
      ms += s;
    }
    fm = block_max(fm, red);
    ms = block_sum(ms, red);
    const float m = fm > -CUDART_INF_F ? fm : 0.f;
    for (int i = threadIdx.x; i < n; i += NT) tc_store_operand(P::exp2(F2[i] - m), vhi, vlo, i);
    if (threadIdx.x == 0) {
      A.mass[p] = ms;
      A.t.Mtgt[p] = m;
    }
  }
}

// ---- FP64 objective of a state on the tensor-core path (gap checks and the returned states) ----
// Per listed problem (CTA = slot): F2 = log2 s - log2 a of the state, with a from the source sums of
// parity `par` (a check: this iteration's), or of the parity of the problem's own last iteration
// (par < 0: the returned states); the target shift M = max F2 and the operand row U = 2^(F2 - M)
// (BF16 hi/lo) of the slot.  Rare, so the row is streamed.
__global__ void __launch_bounds__(256) tc_obj_operand_kernel(TcIterArgs A, const int* list, const int* count,
                                                             int par, float* F2o, float* Mo) {
  using P = Prec<float>;
  __shared__ float red[32];
  const int slot = blockIdx.x;
  if (slot >= *count) return;
  const int p = list[slot], n = A.n;
  const int cur = par >= 0 ? par : (A.iters[p] & 1);
  const float* S = A.S + (size_t)p * n;
  const float* acc = A.t.ACC_src[cur] + (size_t)p * n;
  const float mc = A.t.Msrc[cur][p];
  float* F2 = F2o + (size_t)p * n;
  __nv_bfloat16* vhi = A.t.Vhi + (size_t)slot * A.t.ld;
  __nv_bfloat16* vlo = A.t.Vlo + (size_t)slot * A.t.ld;
  float fm = -CUDART_INF_F;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float sv = S[i];
    const float f2 = sv > 0.f ? P::log2(sv) - tc_log2_sum(acc[i], mc) : P::ninf();
    F2[i] = f2;
    fm = fmaxf(fm, f2);
  }
  fm = block_max(fm, red);  // its barriers also order the F2 writes before the reads below
  const float m = fm > -CUDART_INF_F ? fm : 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tc_store_operand(P::exp2(F2[i] - m), vhi, vlo, i);
  if (threadIdx.x == 0) Mo[p] = m;
}

// The state's target sums (raw, in LB2o) decoded in place to log2 b, and the datafit step g' from
// them (Table 1), for the listed problems.
__global__ void tc_obj_decode_kernel(TcIterArgs A, const int* list, const int* count, float* LB2o, const float* Mo,
                                     float* G2no) {
  const int n = A.n;
  const size_t total = (size_t)(*count) * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int slot = (int)(e / n), j = (int)(e - (size_t)slot * n);
    const int p = list[slot];
    const size_t idx = (size_t)p * n + j;
    const float lb = tc_log2_sum(LB2o[idx], Mo[p]);
    LB2o[idx] = lb;
    G2no[idx] = tc_datafit(A, lb, A.y[idx]);
  }
}

// t = Q^T 1 = 2^{G2 + LB2}, LB2 = Mtgt + log2(target sum); w, g and the per-problem statistics.
__global__ void tc_finalize_kernel(FinArgs<float> F, const float* ACC_tgt, const float* Mtgt) {
  using P = Prec<float>;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t bn = (size_t)F.batch * F.n, bk = (size_t)F.batch * F.k;
  for (size_t e = tid; e < bk; e += stride) F.w_out[e] = F.W[e];
  for (size_t e = tid; e < bn; e += stride) {
    const int p = (int)(e / F.n);
    if (F.g_out) F.g_out[e] = F.G2[e] * F.gscale_inv;
    if (F.t_out) {
      const float lb = tc_log2_sum(ACC_tgt[e], Mtgt[p]);
      F.t_out[e] = lb > -CUDART_INF_F ? P::exp2(F.G2[e] + lb) : 0.f;
    }
  }
  for (size_t e = tid; e < (size_t)F.batch; e += stride) {
    if (F.iters_out) F.iters_out[e] = F.iters[e];
    if (F.status_out) F.status_out[e] = F.status[e];
    if (F.err_out) F.err_out[e] = F.err[e];
  }
}

// Run Algorithm 1 with tensor-core applies and dictionary contractions (float buffers; x, D, y, w,
// g as in solve_device).  Returns cudaErrorLaunchTimeout when a GEMM reported an expired wait.
// ow (may be null when sp.check_every == 0): the objective scratch of the FP64 gap checks.
inline cudaError_t solve_device_tc(const Launch& L, const Workspace<float>& ws, const TcWorkspace& tw,
                                   const TcMMBuf& mb, const ObjWorkspace<float>* ow, const SolveParams& sp,
                                   const float* x, const float* C, const float* D, const float* y, float* w, float* g,
                                   float* t_out, int* iters_out, float* err_out, int* status_out) {
  const int batch = sp.batch, n = sp.n, k = sp.k;
  const double eps_ln2 = sp.eps * kLn2;
  const bool checks = ow && sp.check_every > 0;
  PrepArgs<float> pa;
  pa.x = x; pa.D = D; pa.w_in = w; pa.g_in = g; pa.y = y;
  pa.xt = ws.xt; pa.Dt = ws.Dt; pa.xcol = ws.xcol; pa.W = ws.W; pa.G2 = ws.G2;
  pa.active = ws.active; pa.done = ws.done; pa.n_active = ws.n_active; pa.err_acc = ws.err_acc;
  pa.iters = ws.iters; pa.status = ws.status; pa.err = ws.err;
  pa.dw = ws.dw; pa.all = ws.all; pa.all_count = ws.all_count;
  pa.batch = batch; pa.n = n; pa.k = k;
  pa.xscale = float(grid_scale(sp.cost, eps_ln2));
  pa.gscale = float(1.0 / eps_ln2);
  L.begin(KIND_OTHER);
  prep_kernel<float><<<1184, 256, 0, L.stream>>>(pa);
  L.end();
  L.begin(KIND_OTHER);
  colsum_kernel<float><<<(k + 7) / 8, 256, 0, L.stream>>>(ws.Dt, ws.xcol, n, k);
  L.end();
  L.begin(KIND_OTHER);
  if (C)
    kdense_kernel<<<2048, 256, 0, L.stream>>>(C, n, tw.ld, float(1.0 / eps_ln2), tw.Khi, tw.Klo, tw.Kthi, tw.Ktlo);
  else
    kbuild_kernel<<<2048, 256, 0, L.stream>>>(ws.xt, n, tw.ld, tw.Khi, tw.Klo, sp.cost == COST_ABS);
  L.end();
  L.begin(KIND_OTHER);
  tc_dsplit_kernel<<<1184, 256, 0, L.stream>>>(D, n, k, tw.kp, tw.ld, tw.Dhi, tw.Dlo, tw.Dthi, tw.Dtlo);
  L.end();
  cudaError_t e = cudaMemsetAsync(tw.err, 0, sizeof(int), L.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(tw.hilo, sp.single_until > 0 ? 0 : 0xFF, 2 * sizeof(int), L.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(tw.fix_cnt, 0, 2 * sizeof(unsigned long long), L.stream);
  if (e == cudaSuccess && checks) e = cudaMemsetAsync(ow->kmass, 0, sizeof(double), L.stream);
  if (e != cudaSuccess) return e;
  if (checks) {  // sum_ij K_ij in FP64, once per solve
    L.begin(KIND_OTHER);
    if (C) kernel_mass_dense_kernel<float><<<592, 256, 0, L.stream>>>(C, n, 1.0 / sp.eps, ow->kmass);
    else kernel_mass_kernel<float><<<592, 256, 0, L.stream>>>(x, n, 1.0 / sp.eps, ow->kmass, sp.cost == COST_ABS);
    L.end();
  }

  TcIterArgs ta{};
  ta.active = ws.active; ta.n_active = ws.n_active; ta.n = n; ta.k = k; ta.ld = tw.ld;
  ta.max_iter = sp.max_iter; ta.datafit = sp.datafit; ta.penalty = sp.penalty;
  ta.tol = float(sp.tol); ta.eps = float(sp.eps); ta.alpha = float(sp.alpha); ta.beta = float(sp.beta);
  ta.kl_coef = float(sp.lam / (sp.eps + sp.lam)); ta.tv_bound = float(sp.lam / eps_ln2);
  ta.lam_over_eps = float(sp.lam / sp.eps); ta.log_lam_over_eps = float(log(sp.lam / sp.eps));
  ta.y = y; ta.D = D; ta.Dt = ws.Dt; ta.xcol = ws.xcol; ta.G2 = ws.G2; ta.S = ws.S; ta.F2 = ws.F2; ta.W = ws.W;
  ta.mass = ws.mass; ta.err = ws.err; ta.done = ws.done; ta.iters = ws.iters; ta.status = ws.status; ta.t = tw;
  ta.dw = ws.dw; ta.Wprev = ws.Wprev; ta.dw_tol = float(sp.dw_tol); ta.gap_on = checks && sp.gap_tol > 0;
  ta.gap_ok = checks ? ow->gap_ok : nullptr;
  ta.single_until = float(sp.single_until);

  // the applies K V^T (BF16): M = bins, N = slots mapped to problems, reduction over bins
  tc::GemmArgs ga{};
  ga.col_map = ws.active; ga.n_cols = ws.n_active; ga.M = n; ga.N = batch; ga.Kd = n; ga.ld_out = n;
  ga.err = tw.err; ga.fix_list = tw.fix_list; ga.fix_cap = (unsigned long long)batch * n; ga.splits = 1;
  ga.hilo = tw.hilo;
  {
    const int units = ((n + tc::BM - 1) / tc::BM) * ((batch + tc::BN - 1) / tc::BN);
    if (batch <= TC_SMALL_BATCH && units < tc::num_sms()) {
      ga.splits = tc::choose_splits(units, (n + tc::KindTraits<tc::KIND_BF16>::BK - 1) / tc::KindTraits<tc::KIND_BF16>::BK);
      if (ga.splits > TC_APPLY_SPLITS) ga.splits = TC_APPLY_SPLITS;
    }
    ga.split_stride = (size_t)batch * n;
    if (ga.splits > 1) ga.fix_list = nullptr;  // listed by tc_split_reduce_kernel instead
  }
  const int abs_cost = sp.cost == COST_ABS;
  const TcCost cost_src{ws.xt, C, float(1.0 / eps_ln2), 0, abs_cost}, cost_tgt{ws.xt, C, float(1.0 / eps_ln2), 1, abs_cost};
  const int red_grid = (int)(((size_t)batch * n + 255) / 256 < 1184 ? ((size_t)batch * n + 255) / 256 : 1184);
  // the BF16 GEMM of an apply: the two-SM kernel (256 x 128 tiles over SM pairs) when the reduction
  // is not split, else the one-SM kernel with its split partial sums
  auto launch_apply = [&](const __nv_bfloat16* Ah, const __nv_bfloat16* Al, const __nv_bfloat16* Bh,
                          const __nv_bfloat16* Bl, const tc::GemmArgs& a) -> cudaError_t {
    if (a.splits == 1) return tc::launch_gemm3_pair<tc::KIND_BF16>(Ah, Al, tw.ld, Bh, Bl, tw.ld, n, batch, n, a, L.stream);
    return tc::launch_gemm3<tc::KIND_BF16>(Ah, Al, tw.ld, Bh, Bl, tw.ld, n, batch, n, a, L.stream);
  };
  // one apply into `acc` (counting underflows into `cnt`): split partial sums are added afterwards
  // the source apply reads K, the target apply K^T (the same matrix for the symmetric grid cost)
  auto apply = [&](float* acc, unsigned long long* cnt, bool target) -> cudaError_t {
    ga.out = ga.splits > 1 ? tw.ACCP : acc;
    ga.fix_cnt = cnt;
    const bool kt = target && C;
    L.begin(KIND_APPLY);
    cudaError_t r = launch_apply(kt ? tw.Kthi : tw.Khi, kt ? tw.Ktlo : tw.Klo, tw.Vhi, tw.Vlo, ga);
    if (r == cudaSuccess && ga.splits > 1) {
      tc_split_reduce_kernel<<<red_grid, 256, 0, L.stream>>>(tw.ACCP, ga.splits, ga.split_stride, ws.active,
                                                              ws.n_active, n, acc, tw.fix_list, cnt, ga.fix_cap);
      r = cudaGetLastError();
    }
    L.end();
    return r;
  };
  // D^T r (TF32): M = dictionary columns, N = slots (partial sums by slot), reduction over bins split
  tc::GemmArgs gr{};
  gr.out = mb.NU; gr.n_cols = ws.n_active; gr.M = k; gr.N = batch; gr.Kd = n; gr.ld_out = mb.ldnu; gr.err = tw.err;
  gr.splits = tc::choose_splits(((k + tc::BM - 1) / tc::BM) * ((batch + tc::BN - 1) / tc::BN),
                                (n + tc::KindTraits<tc::KIND_TF32>::BK - 1) / tc::KindTraits<tc::KIND_TF32>::BK);
  gr.split_stride = mb.plane;
  // s = D w (TF32, two-SM kernel): M = bins, N = slots mapped to problems, reduction over dictionary
  // columns
  tc::GemmArgs gw{};
  gw.out = ws.S; gw.col_map = ws.active; gw.n_cols = ws.n_active; gw.M = n; gw.N = batch; gw.Kd = k;
  gw.ld_out = n; gw.err = tw.err; gw.flush_tiny = 1; gw.splits = 1; gw.store_direct = 1;
  const int row_cfg = tc_row_cfg(n);

  // FP64 objective of the listed problems' states (w, g) on the tensor-core applies: the state's
  // source sums (parity par, or each problem's last when par < 0) give F2, one target GEMM of its
  // operand (into the objective scratch, with its own fix-up list count) gives b and g', then the
  // FP64 reduction; gap = true also records the gap test.
  auto objective_tc = [&](const int* list, const int* count, int par, bool gap) -> cudaError_t {
    L.begin(KIND_OTHER);
    tc_obj_operand_kernel<<<batch, 256, 0, L.stream>>>(ta, list, count, par, ow->F2, ow->M);
    L.end();
    cudaError_t r = cudaMemsetAsync(tw.fix_cnt + 2, 0, sizeof(unsigned long long), L.stream);
    if (r != cudaSuccess) return r;
    tc::GemmArgs go = ga;
    go.col_map = list; go.n_cols = count; go.fix_cnt = tw.fix_cnt + 2;
    go.hilo = nullptr;  // the objective's apply always takes the three products
    go.out = go.splits > 1 ? tw.ACCP : ow->LB2;
    L.begin(KIND_APPLY);
    r = launch_apply(C ? tw.Kthi : tw.Khi, C ? tw.Ktlo : tw.Klo, tw.Vhi, tw.Vlo, go);
    if (r == cudaSuccess && go.splits > 1) {
      tc_split_reduce_kernel<<<red_grid, 256, 0, L.stream>>>(tw.ACCP, go.splits, go.split_stride, list, count, n,
                                                              ow->LB2, tw.fix_list, tw.fix_cnt + 2, go.fix_cap);
      r = cudaGetLastError();
    }
    L.end();
    if (r != cudaSuccess) return r;
    L.begin(KIND_OTHER);
    tc_fixup_kernel<<<TC_FIX_GRID, 256, 0, L.stream>>>(tw.fix_list, tw.fix_cnt + 2, tw.fix_cnt + 3, ga.fix_cap, n,
                                                    cost_tgt, ow->F2, ow->LB2, ow->M);
    L.end();
    L.begin(KIND_OTHER);
    tc_obj_decode_kernel<<<red_grid, 256, 0, L.stream>>>(ta, list, count, ow->LB2, ow->M, ow->G2n);
    L.end();
    ObjArgs<float> oa = obj_args<float>(sp, D, ws.xcol, ws.W, y, ws.S, ws.G2, *ow);
    oa.list = list; oa.count = count; oa.gap_ok = gap ? ow->gap_ok : nullptr;
    L.begin(KIND_OTHER);
    objective_reduce_kernel<float><<<batch, 256, 0, L.stream>>>(oa);
    L.end();
    return cudaGetLastError();
  };

  // the initial source marginal s = D w0, through the same operand and GEMM as every iteration
  // (the mass sum_i s_i is first needed by the violation at it = 1 and set by the operand kernel)
  L.begin(KIND_OTHER);
  tc_wupd_kernel<<<(int)(((long long)batch * k + 255) / 256), 256, 0, L.stream>>>(ta, mb, 0, 0, 0);
  L.end();
  L.begin(KIND_OTHER);
  e = tc::launch_gemm3_pair<tc::KIND_TF32>(tw.Dhi, tw.Dlo, tw.kp, tw.Whi, tw.Wlo, tw.kp, n, batch, k, gw, L.stream);
  L.end();
  if (e != cudaSuccess) return e;

  for (int it = 0;; ++it) {
    ta.it = it;
    L.begin(KIND_MM);
    TC_ROW_LAUNCH(tc_prep_src_kernel, row_cfg, batch, L.stream, ta);
    L.end();
    e = apply(tw.ACC_src[it & 1], tw.fix_cnt, false);
    if (e != cudaSuccess) return e;
    L.begin(KIND_OTHER);
    tc_fixup_kernel<<<TC_FIX_GRID, 256, 0, L.stream>>>(tw.fix_list, tw.fix_cnt, tw.fix_cnt + 1, ga.fix_cap, n,
                                                    cost_src, ws.G2, tw.ACC_src[it & 1], tw.Msrc[it & 1]);
    L.end();
    // a check: the state (w, g) whose source sums were just computed is the one this iteration
    // returns if it stops here; its FP64 objective and gap come before the stopping decision
    const bool check = checks && it > 0 && it % sp.check_every == 0;
    if (check) {
      e = objective_tc(ws.active, ws.n_active, it & 1, true);
      if (e != cudaSuccess) return e;
    }
    ta.gap_check = check;
    L.begin(KIND_MM);
    TC_ROW_LAUNCH(tc_violation_kernel, row_cfg, batch, L.stream, ta);
    L.end();
    if (it >= sp.max_iter) break;
    L.begin(KIND_MM);
    e = tc::launch_gemm3<tc::KIND_TF32>(tw.Dthi, tw.Dtlo, tw.ld, tw.Rhi, tw.Rlo, tw.ld, k, batch, n, gr, L.stream);
    L.end();
    if (e != cudaSuccess) return e;
    L.begin(KIND_MM);
    tc_wupd_kernel<<<(int)(((long long)batch * k + 255) / 256), 256, 0, L.stream>>>(ta, mb, gr.splits, 1, 1);
    L.end();
    L.begin(KIND_MM);
    e = tc::launch_gemm3_pair<tc::KIND_TF32>(tw.Dhi, tw.Dlo, tw.kp, tw.Whi, tw.Wlo, tw.kp, n, batch, k, gw, L.stream);
    L.end();
    if (e != cudaSuccess) return e;
    // further MM steps with the same a: log ratios from the new s, D^T r, update, s = D w
    for (int m = 1; m < sp.mm_steps; ++m) {
      L.begin(KIND_MM);
      TC_ROW_LAUNCH(tc_ratio_kernel, row_cfg, batch, L.stream, ta);
      L.end();
      L.begin(KIND_MM);
      e = tc::launch_gemm3<tc::KIND_TF32>(tw.Dthi, tw.Dtlo, tw.ld, tw.Rhi, tw.Rlo, tw.ld, k, batch, n, gr, L.stream);
      L.end();
      if (e != cudaSuccess) return e;
      L.begin(KIND_MM);
      tc_wupd_kernel<<<(int)(((long long)batch * k + 255) / 256), 256, 0, L.stream>>>(ta, mb, gr.splits, 1, 0);
      L.end();
      L.begin(KIND_MM);
      e = tc::launch_gemm3_pair<tc::KIND_TF32>(tw.Dhi, tw.Dlo, tw.kp, tw.Whi, tw.Wlo, tw.kp, n, batch, k, gw, L.stream);
      L.end();
      if (e != cudaSuccess) return e;
    }
    if (it > 0) {
      L.begin(KIND_COMPACT);
      compact_kernel<<<1, 1024, 0, L.stream>>>(ws.active, ws.n_active, ws.done);
      L.end();
    }
    L.begin(KIND_MM);
    TC_ROW_LAUNCH(tc_operand_kernel, row_cfg, batch, L.stream, ta);
    L.end();
    e = apply(tw.ACC_tgt, tw.fix_cnt + 1, true);
    if (e != cudaSuccess) return e;
    L.begin(KIND_OTHER);
    tc_fixup_kernel<<<TC_FIX_GRID, 256, 0, L.stream>>>(tw.fix_list, tw.fix_cnt + 1, tw.fix_cnt, ga.fix_cap, n,
                                                    cost_tgt, ws.F2, tw.ACC_tgt, tw.Mtgt);
    L.end();
    if ((it + 1) % sp.poll_every == 0) {
      e = cudaMemcpyAsync(L.host_flag, ws.n_active, sizeof(int), cudaMemcpyDeviceToHost, L.stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
      if (e == cudaSuccess && L.timer && L.timer->on) e = L.timer->harvest();
      if (e != cudaSuccess) return e;
      if (*L.host_flag == 0) break;
    }
  }
  // the returned states' objective (every problem's last source sums are those of its final g)
  if (checks) {
    e = objective_tc(ws.all, ws.all_count, -1, false);
    if (e != cudaSuccess) return e;
  }
  FinArgs<float> fa;
  fa.W = ws.W; fa.G2 = ws.G2; fa.LB2 = nullptr; fa.iters = ws.iters; fa.status = ws.status; fa.err = ws.err;
  fa.w_out = w; fa.g_out = g; fa.t_out = t_out; fa.iters_out = iters_out; fa.status_out = status_out;
  fa.err_out = err_out; fa.batch = batch; fa.n = n; fa.k = k; fa.gscale_inv = float(eps_ln2);
  L.begin(KIND_OTHER);
  tc_finalize_kernel<<<1184, 256, 0, L.stream>>>(fa, tw.ACC_tgt, tw.Mtgt);
  L.end();
  e = cudaMemcpyAsync(L.host_flag, tw.err, sizeof(int), cudaMemcpyDeviceToHost, L.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
  if (e == cudaSuccess && L.timer && L.timer->on) e = L.timer->harvest();
  if (e != cudaSuccess) return e;
  return *L.host_flag ? cudaErrorLaunchTimeout : cudaGetLastError();
}

}  // namespace otlm
