// Kernels of the batched OTLM scaling iteration (Algorithm 1) on a shared 1-D grid and a shared
// dictionary, carried in the log domain:
//   G2 = g / (eps ln2)   target potential,  F2 = f / (eps ln2)   source potential,
//   LA2 = log2 (K u1),  LB2 = log2 (K^T u2),  S = X w  (the paper's X is the dictionary D).
// With the scaled grid xt = x / sqrt(eps ln2), C_ij / (eps ln2) = (xt_i - xt_j)^2, so
//   LA2_i = log2 sum_j 2^(G2_j - (xt_i - xt_j)^2),   LB2_j = log2 sum_i 2^(F2_i - (xt_i - xt_j)^2).
// The absolute-distance grid cost C_ij = |x_i - x_j| (the cost of the paper's demonstrations and
// scalability tests, there scaled by rho: pass rho x) takes xt = x / (eps ln2) and |xt_i - xt_j|.
// A dense cost C [n][n] (any, e.g. non-symmetric or truncated with +inf) is read in tiles: the
// source apply sums along row i of C, the target apply along column j, in units C / (eps ln2).
#pragma once

#include "common.cuh"

namespace otlm {

enum { EPI_SOURCE = 0, EPI_TARGET = 1 };
enum { COST_SQ = 0, COST_ABS = 1, COST_DENSE = 2 };  // (xt_i - xt_j)^2, |xt_i - xt_j|, or C_ij / (eps ln2)

template <int COST, typename T>
__device__ __forceinline__ T grid_cost(T d) {
  if constexpr (COST == COST_ABS) return fabs(d);
  else return d * d;
}
enum { DF_BALANCED = 0, DF_KL = 1, DF_TV = 2, DF_L2 = 3, DF_POISSON = 4 };
enum { PEN_NONE = 0, PEN_L1 = 1, PEN_L2SQ = 2, PEN_ELASTIC = 3 };
enum { ST_CONVERGED = 0, ST_MAX_ITER = 1, ST_NONFINITE = 2, ST_INVALID = 3 };

// Poisson datafit step (reading A7) in log2 units, from v = log2 b and the target bin y:
// G2 = log2(lam y/eps) - log2 omega(ln(lam y/eps) - ln b + lam/eps) - v, and -lam/(eps ln2) where
// y = 0 (`neg_bound`).  Kept out of line so that the apply kernel's epilogue keeps its registers.
template <typename T>
__device__ __noinline__ T poisson_g2(T log_lam_over_eps, T lam_over_eps, T neg_bound, T v, T yv) {
  using P = Prec<T>;
  if (!(yv > T(0))) return -neg_bound;
  const T l2c = log_lam_over_eps * T(kLog2e) + P::log2(yv);
  return l2c - P::log2(wright_omega<T>((l2c - v) * T(kLn2) + lam_over_eps)) - v;
}

template <typename T>
struct ApplyArgs {
  const T* in;          // [P][n] potentials in log2 units (G2 for the source apply, F2 for the target apply)
  T* out;               // [P][n] log2 sums; on entry the previous sums (the fast path's shift)
  const T* xt;          // [n] scaled grid
  const int* active;    // active problem ids, compacted
  const int* n_active;  // number of active problems
  int n;
  // source-apply epilogue: violation e = sum_i S_i |2^(LA2new_i - LA2old_i) - 1| (numerator)
  const T* S;           // [P][n] X w of the previous source step
  T* err_acc;           // [P] numerators, accumulated atomically
  int check;
  // target-apply epilogue: datafit prox (Table 1) in log2 units
  const T* y;           // [P][n]
  T* G2;                // [P][n]
  int datafit;
  T kl_coef;            // lam / (eps + lam)
  T tv_bound;           // lam / (eps ln2)
  T lam_over_eps;       // lam / eps
  T log_lam_over_eps;   // ln(lam / eps)
  // dense cost (the COST_DENSE kernels): C [n][n] row-major, the source apply reading row i (the
  // output row) and the target apply (c_trans = 1) column j; scaled by c_scale = 1 / (eps ln2)
  const T* C;
  T c_scale;
  int c_trans;
};

// Tile of the kernel apply: TB = RB*WB problems x TI = 32*RI*WI rows; warp (wb, wi) owns RB
// problems and 32*RI rows, lane l the rows wi*32*RI + r*32 + l.  The input potentials of the
// CTA's problems are staged through shared memory in chunks of TJ columns, stored [j][b] so that
// every lane reads its RB problems of one column as one broadcast vector load.
template <typename T, int RB_, int RI_, int WB_, int WI_, int TJ_>
struct ApplyTile {
  static constexpr int RB = RB_, RI = RI_, WB = WB_, WI = WI_, TJ = TJ_;
  static constexpr int TB = RB * WB, TI = 32 * RI * WI, NT = 32 * WB * WI;
};

enum { SHIFT_PREV = 0, SHIFT_DIAG = 1, SHIFT_EXACT = 2 };

template <typename T, int N> struct VecLoad;  // N consecutive T from shared memory
template <> struct VecLoad<float, 4> {
  static __device__ __forceinline__ void ld(const float* p, float* v) {
    float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
};
template <> struct VecLoad<double, 2> {
  static __device__ __forceinline__ void ld(const double* p, double* v) {
    double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x; v[1] = q.y;
  }
};

// Packed FP32x2 arithmetic (two lanes of a 64-bit register per instruction).
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// Dense-cost tile of a chunk, c_s[jj][il] (row pitch TI + 1) = C2 of output row i0 + il and summed
// index j0 + jj: C[i][j] for the source apply (read along j, transposed into shared memory), C[j][i]
// for the target apply (read along i); +inf outside [0, n), so that the term vanishes.
template <typename T, class Cfg>
__device__ __forceinline__ void stage_cost_tile(const ApplyArgs<T>& A, T* c_s, int i0, int j0) {
  constexpr int TI = Cfg::TI, TJ = Cfg::TJ, NT = Cfg::NT, TIP = TI + 1;
  const int n = A.n;
  const T inf = -Prec<T>::ninf();
  for (int e = threadIdx.x; e < TI * TJ; e += NT) {
    if (!A.c_trans) {  // consecutive threads: consecutive j of one row i
      const int il = e / TJ, jj = e - il * TJ, i = i0 + il, j = j0 + jj;
      c_s[jj * TIP + il] = (i < n && j < n) ? A.C[(size_t)i * n + j] * A.c_scale : inf;
    } else {  // consecutive threads: consecutive i of one row j of C
      const int jj = e / TI, il = e - jj * TI, i = i0 + il, j = j0 + jj;
      c_s[jj * TIP + il] = (i < n && j < n) ? A.C[(size_t)j * n + i] * A.c_scale : inf;
    }
  }
}

// Stage one chunk of TJ columns: the CTA's TB input rows into in_s[j][b] and the grid values (or,
// for a dense cost, the cost tile).
template <typename T, class Cfg, int COST>
__device__ __forceinline__ void stage_chunk(const ApplyArgs<T>& A, const int* prob_s, T* in_s, T* xj_s, T* c_s,
                                            int i0, int j0) {
  using P = Prec<T>;
  constexpr int TB = Cfg::TB, TJ = Cfg::TJ, NT = Cfg::NT;
  const int n = A.n;
  __syncthreads();
  for (int e = threadIdx.x; e < TB * TJ; e += NT) {
    const int bb = e / TJ, jj = e - bb * TJ, j = j0 + jj, p = prob_s[bb];
    in_s[jj * TB + bb] = (p >= 0 && j < n) ? A.in[(size_t)p * n + j] : P::ninf();
  }
  if constexpr (COST == COST_DENSE) stage_cost_tile<T, Cfg>(A, c_s, i0, j0);
  else
    for (int jj = threadIdx.x; jj < TJ; jj += NT) xj_s[jj] = (j0 + jj < n) ? A.xt[j0 + jj] : T(0);
  __syncthreads();
}

// Exact shift: m = max_j (in_bj - c_ij), c_ij the grid cost (scalar; the rare path).
// The cost of term jj for row r: the grid cost of xi[r] - xj, or the dense tile's entry of the
// thread's row il0 + 32 r.
template <typename T, class Cfg, int COST>
__device__ __forceinline__ T term_cost(const T (&xi)[Cfg::RI], T xj, const T* c_s, int il0, int jj, int r) {
  if constexpr (COST == COST_DENSE) return c_s[jj * (Cfg::TI + 1) + il0 + 32 * r];
  else return grid_cost<COST>(xi[r] - xj);
}

template <typename T, class Cfg, int COST>
__device__ __forceinline__ void sweep_max(const ApplyArgs<T>& A, const int* prob_s, T* in_s, T* xj_s, T* c_s, int i0,
                                          int il0, const T (&xi)[Cfg::RI], int wb, T (&m)[Cfg::RB][Cfg::RI]) {
  constexpr int RB = Cfg::RB, RI = Cfg::RI, TB = Cfg::TB, TJ = Cfg::TJ;
  for (int j0 = 0; j0 < A.n; j0 += TJ) {
    stage_chunk<T, Cfg, COST>(A, prob_s, in_s, xj_s, c_s, i0, j0);
#pragma unroll 4
    for (int jj = 0; jj < TJ; ++jj) {
      const T xj = COST == COST_DENSE ? T(0) : xj_s[jj];
      T v[RB];
      VecLoad<T, RB>::ld(in_s + jj * TB + wb * RB, v);
#pragma unroll
      for (int r = 0; r < RI; ++r) {
        const T c = term_cost<T, Cfg, COST>(xi, xj, c_s, il0, jj, r);
#pragma unroll
        for (int q = 0; q < RB; ++q) m[q][r] = fmax(m[q][r], v[q] - c);
      }
    }
  }
}

// Sum with a known shift: acc = sum_j 2^(in_bj - m_bi - c_ij).  Generic (double) version.
template <typename T, class Cfg, int COST>
__device__ __forceinline__ void sweep_sum(const ApplyArgs<T>& A, const int* prob_s, T* in_s, T* xj_s, T* c_s, int i0,
                                          int il0, const T (&xi)[Cfg::RI], int wb, const T (&m)[Cfg::RB][Cfg::RI],
                                          T (&acc)[Cfg::RB][Cfg::RI]) {
  using P = Prec<T>;
  constexpr int RB = Cfg::RB, RI = Cfg::RI, TB = Cfg::TB, TJ = Cfg::TJ;
  for (int j0 = 0; j0 < A.n; j0 += TJ) {
    stage_chunk<T, Cfg, COST>(A, prob_s, in_s, xj_s, c_s, i0, j0);
#pragma unroll 4
    for (int jj = 0; jj < TJ; ++jj) {
      const T xj = COST == COST_DENSE ? T(0) : xj_s[jj];
      T v[RB];
      VecLoad<T, RB>::ld(in_s + jj * TB + wb * RB, v);
#pragma unroll
      for (int r = 0; r < RI; ++r) {
        const T d = xi[r] - xj;
#pragma unroll
        for (int q = 0; q < RB; ++q) {
          if constexpr (COST == COST_DENSE) acc[q][r] += P::exp2((v[q] - m[q][r]) - c_s[jj * (Cfg::TI + 1) + il0 + 32 * r]);
          else if constexpr (COST == COST_ABS) acc[q][r] += P::exp2((v[q] - m[q][r]) - fabs(d));
          else acc[q][r] += P::exp2(fma(-d, d, v[q] - m[q][r]));
        }
      }
    }
  }
}

// FP32 path: centred expansion.  With a tile centre xc, di = xt_i - xc and dj = xt_j - xc,
//   in_bj - m_bi - (xt_i - xt_j)^2 = h_bj + 2 di dj - q_bi,   h_bj = in_bj - dj^2,  q_bi = m_bi + di^2.
// h is formed once per staged element, q once per row, so an element costs one FFMA and one FADD
// plus the accumulate: on packed pairs of problems (fma/add.f32x2) that is three FP32 lane-ops per
// element against one exponent-unit op, and the exponent unit (32 results / SM / clock) is the
// bound.  The centre keeps di small (a tile spans TI rows) and dj is small for every column that
// matters, so no large squares are added and cancelled.
// Absolute-distance cost (COST_ABS): no expansion; the staged values are the inputs themselves and
// the grid values xt_j, and an element costs the difference xt_i - xt_j (shared by a packed pair of
// problems) and two packed adds.
template <class Cfg, int COST>
__device__ __forceinline__ void stage_chunk_f32(const ApplyArgs<float>& A, const int* prob_s, float* h_s, float* dj_s,
                                                float xc, int j0) {
  using P = Prec<float>;
  constexpr int TB = Cfg::TB, TJ = Cfg::TJ, NT = Cfg::NT;
  const int n = A.n;
  __syncthreads();
  for (int jj = threadIdx.x; jj < TJ; jj += NT) {
    const float d = (j0 + jj < n) ? (COST == COST_ABS ? A.xt[j0 + jj] : A.xt[j0 + jj] - xc) : 0.f;
    dj_s[2 * jj] = d;
    dj_s[2 * jj + 1] = d;
  }
  for (int e = threadIdx.x; e < TB * TJ; e += NT) {
    const int bb = e / TJ, jj = e - bb * TJ, j = j0 + jj, p = prob_s[bb];
    float h = P::ninf();
    if (p >= 0 && j < n) {
      if constexpr (COST == COST_ABS) {
        h = A.in[(size_t)p * n + j];
      } else {
        const float d = A.xt[j] - xc;
        h = fmaf(-d, d, A.in[(size_t)p * n + j]);
      }
    }
    h_s[jj * TB + bb] = h;
  }
  __syncthreads();
}

template <class Cfg, int COST>
__device__ __forceinline__ void sweep_max_f32(const ApplyArgs<float>& A, const int* prob_s, float* h_s, float* dj_s,
                                              float xc, const float (&xi)[Cfg::RI], const float (&di)[Cfg::RI],
                                              int wb, float (&m)[Cfg::RB][Cfg::RI]) {
  constexpr int RB = Cfg::RB, RI = Cfg::RI, TB = Cfg::TB, TJ = Cfg::TJ;
  for (int j0 = 0; j0 < A.n; j0 += TJ) {
    stage_chunk_f32<Cfg, COST>(A, prob_s, h_s, dj_s, xc, j0);
#pragma unroll 4
    for (int jj = 0; jj < TJ; ++jj) {
      const float dj = dj_s[2 * jj];
      float h[RB];
      VecLoad<float, RB>::ld(h_s + jj * TB + wb * RB, h);
#pragma unroll
      for (int r = 0; r < RI; ++r)
#pragma unroll
        for (int q = 0; q < RB; ++q) {
          if constexpr (COST == COST_ABS) m[q][r] = fmaxf(m[q][r], h[q] - fabsf(xi[r] - dj));
          else m[q][r] = fmaxf(m[q][r], fmaf(2.f * di[r], dj, h[q]));
        }
    }
  }
  if constexpr (COST == COST_SQ) {
#pragma unroll
    for (int r = 0; r < RI; ++r)
#pragma unroll
      for (int q = 0; q < RB; ++q) m[q][r] -= di[r] * di[r];
  }
}

template <class Cfg, int COST>
__device__ __forceinline__ void sweep_sum_f32(const ApplyArgs<float>& A, const int* prob_s, float* h_s, float* dj_s,
                                              float xc, const float (&xi)[Cfg::RI], const float (&di)[Cfg::RI],
                                              int wb, const float (&m)[Cfg::RB][Cfg::RI],
                                              float (&acc)[Cfg::RB][Cfg::RI]) {
  using P = Prec<float>;
  constexpr int RB = Cfg::RB, RI = Cfg::RI, TB = Cfg::TB, TJ = Cfg::TJ, QP = RB / 2;
  static_assert(RB == 4, "packed sweep expects 4 problems per thread");
  uint64_t nq[QP][RI], acc2[QP][RI], tdi[RI];
#pragma unroll
  for (int r = 0; r < RI; ++r) {
    tdi[r] = f2_pack(2.f * di[r], 2.f * di[r]);
    const float d2 = COST == COST_ABS ? 0.f : di[r] * di[r];
#pragma unroll
    for (int p = 0; p < QP; ++p) {
      nq[p][r] = f2_pack(-(m[2 * p][r] + d2), -(m[2 * p + 1][r] + d2));
      acc2[p][r] = f2_pack(0.f, 0.f);
    }
  }
  for (int j0 = 0; j0 < A.n; j0 += TJ) {
    stage_chunk_f32<Cfg, COST>(A, prob_s, h_s, dj_s, xc, j0);
#pragma unroll 4
    for (int jj = 0; jj < TJ; ++jj) {
      const float2 dq = *reinterpret_cast<const float2*>(dj_s + 2 * jj);
      const float4 hq = *reinterpret_cast<const float4*>(h_s + jj * TB + wb * RB);
      const uint64_t dj2 = f2_pack(dq.x, dq.y);
      const uint64_t h2[QP] = {f2_pack(hq.x, hq.y), f2_pack(hq.z, hq.w)};
#pragma unroll
      for (int r = 0; r < RI; ++r) {
        uint64_t nad = 0;  // -|xt_i - xt_j| on both lanes (absolute-distance cost)
        if constexpr (COST == COST_ABS) {
          const float ad = -fabsf(xi[r] - dq.x);
          nad = f2_pack(ad, ad);
        }
#pragma unroll
        for (int p = 0; p < QP; ++p) {
          const uint64_t u2 = COST == COST_ABS ? f2_add(f2_add(h2[p], nq[p][r]), nad)
                                               : f2_add(f2_fma(tdi[r], dj2, h2[p]), nq[p][r]);
          float u0, u1;
          f2_unpack(u2, u0, u1);
          acc2[p][r] = f2_add(acc2[p][r], f2_pack(P::exp2(u0), P::exp2(u1)));
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RI; ++r)
#pragma unroll
    for (int p = 0; p < QP; ++p) f2_unpack(acc2[p][r], acc[2 * p][r], acc[2 * p + 1][r]);
}

// Kernel apply with fused epilogue.  The sum needs a shift m_bi close to the result:
//   SHIFT_PREV : the previous sums held in `out` (the iteration after the first),
//   SHIFT_DIAG : the diagonal term in_bi (c_ii = 0, so every sum is >= 1; the first iteration),
//   SHIFT_EXACT: an exact max pass first.
// A fast shift is checked afterwards: if any sum of the tile leaves [2^-60, 2^60] (or a shift is
// not finite) the CTA redoes its tile with the exact shift.
template <typename T, class Cfg, int EPI, int SHIFT, int COST>
__global__ void __launch_bounds__(Cfg::NT) apply_kernel(ApplyArgs<T> A) {
  using P = Prec<T>;
  constexpr int RB = Cfg::RB, RI = Cfg::RI, WB = Cfg::WB, TB = Cfg::TB, TI = Cfg::TI, TJ = Cfg::TJ;
  __shared__ __align__(16) T in_s[TJ * TB];
  __shared__ __align__(16) T xj_s[2 * TJ];
  __shared__ T c_s[COST == COST_DENSE ? TJ * (TI + 1) : 1];
  __shared__ int prob_s[TB];
  const int na = *A.n_active;
  const int b0 = blockIdx.y * TB;
  if (b0 >= na) return;
  const int n = A.n;
  const int i0 = blockIdx.x * TI;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wb = warp % WB, wi = warp / WB;
  if (threadIdx.x < TB) prob_s[threadIdx.x] = (b0 + threadIdx.x < na) ? A.active[b0 + threadIdx.x] : -1;
  __syncthreads();
  int pr[RB];
#pragma unroll
  for (int q = 0; q < RB; ++q) pr[q] = prob_s[wb * RB + q];
  int row[RI];
  T xi[RI], di[RI];
  // tile centre for the FP32 expansion (any value is exact in real arithmetic; the middle of the
  // tile keeps the squares small)
  const T xc = COST == COST_DENSE ? T(0) : T(0.5) * (A.xt[min(i0, n - 1)] + A.xt[min(i0 + TI - 1, n - 1)]);
  const int il0 = wi * 32 * RI + lane;  // the thread's first row within the tile (dense-cost tiles)
#pragma unroll
  for (int r = 0; r < RI; ++r) {
    row[r] = i0 + il0 + r * 32;
    xi[r] = (COST != COST_DENSE && row[r] < n) ? A.xt[row[r]] : xc;
    di[r] = xi[r] - xc;
  }
  T m[RB][RI], acc[RB][RI];
  bool safe = SHIFT == SHIFT_EXACT;
  if (!safe) {
    const T* src = SHIFT == SHIFT_PREV ? A.out : A.in;
    bool bad = false;
#pragma unroll
    for (int q = 0; q < RB; ++q)
#pragma unroll
      for (int r = 0; r < RI; ++r) {
        const bool ok = pr[q] >= 0 && row[r] < n;
        m[q][r] = ok ? src[(size_t)pr[q] * n + row[r]] : T(0);
        acc[q][r] = T(0);
        bad |= ok && !isfinite(m[q][r]);
      }
    safe = __syncthreads_or(bad);
    if (!safe) {
      if constexpr (sizeof(T) == 4 && COST != COST_DENSE)
        sweep_sum_f32<Cfg, COST>(A, prob_s, in_s, xj_s, xc, xi, di, wb, m, acc);
      else sweep_sum<T, Cfg, COST>(A, prob_s, in_s, xj_s, c_s, i0, il0, xi, wb, m, acc);
      bad = false;
#pragma unroll
      for (int q = 0; q < RB; ++q)
#pragma unroll
        for (int r = 0; r < RI; ++r) {
          const bool ok = pr[q] >= 0 && row[r] < n;
          bad |= ok && !(acc[q][r] >= T(8.673617379884035e-19) && acc[q][r] <= T(1.152921504606847e18));
        }
      safe = __syncthreads_or(bad);
    }
  }
  if (safe) {
#pragma unroll
    for (int q = 0; q < RB; ++q)
#pragma unroll
      for (int r = 0; r < RI; ++r) { m[q][r] = P::ninf(); acc[q][r] = T(0); }
    if constexpr (sizeof(T) == 4 && COST != COST_DENSE) sweep_max_f32<Cfg, COST>(A, prob_s, in_s, xj_s, xc, xi, di, wb, m);
    else sweep_max<T, Cfg, COST>(A, prob_s, in_s, xj_s, c_s, i0, il0, xi, wb, m);
#pragma unroll
    for (int q = 0; q < RB; ++q)
#pragma unroll
      for (int r = 0; r < RI; ++r)
        if (!(m[q][r] > P::ninf())) m[q][r] = T(0);  // every term vanishes: the sum stays 0
    if constexpr (sizeof(T) == 4 && COST != COST_DENSE)
      sweep_sum_f32<Cfg, COST>(A, prob_s, in_s, xj_s, xc, xi, di, wb, m, acc);
    else sweep_sum<T, Cfg, COST>(A, prob_s, in_s, xj_s, c_s, i0, il0, xi, wb, m, acc);
  }
  const bool prev_shift = SHIFT == SHIFT_PREV && !safe;  // then acc = a_new / a_old exactly

  // ---- epilogue -----------------------------------------------------------------------------
#pragma unroll
  for (int q = 0; q < RB; ++q) {
    const int p = pr[q];
    T part = T(0);
    if (p >= 0) {
#pragma unroll
      for (int r = 0; r < RI; ++r) {
        if (row[r] >= n) continue;
        const size_t idx = (size_t)p * n + row[r];
        const T v = acc[q][r] > T(0) ? m[q][r] + P::log2(acc[q][r]) : P::ninf();
        if (EPI == EPI_SOURCE) {
          if (A.check) {
            // s |a_new / a_old - 1| = s |2^dl - 1|: expm1 keeps the small ratios (the ones that
            // decide convergence) accurate; a jump beyond 2^64 is taken in log form, capped at
            // 2^120, so that an early, far-off row cannot overflow to inf.
            // On the fast path the shift m is the previous LA2 itself, so the ratio a_new/a_old is
            // the tile sum acc, known to FP32 relative precision; subtracting two logs of size
            // |LA2| would quantise it to |LA2| ulp.
            const T s = A.S[idx];
            if (s > T(0)) {
              if (prev_shift) {
                part += s * fabs(acc[q][r] - T(1));
              } else {
                const T dl = v - A.out[idx];
                part += dl > T(64) ? P::exp2(fmin(P::log2(s) + dl, T(120))) : s * fabs(P::expm1(dl * T(kLn2)));
              }
            }
          }
          A.out[idx] = v;
        } else {
          A.out[idx] = v;
          const T yv = A.y[idx];
          T gn;
          switch (A.datafit) {
            case DF_BALANCED: gn = P::log2(yv) - v; break;
            case DF_KL: gn = A.kl_coef * (P::log2(yv) - v); break;
            case DF_TV: gn = fmin(fmax(P::log2(yv) - v, -A.tv_bound), A.tv_bound); break;
            case DF_POISSON: gn = poisson_g2<T>(A.log_lam_over_eps, A.lam_over_eps, A.tv_bound, v, yv); break;
            default: {  // L2: g = lam y - eps omega(ln(lam/eps) + ln b + (lam/eps) y)
              const T z = A.log_lam_over_eps + v * T(kLn2) + A.lam_over_eps * yv;
              gn = (A.lam_over_eps * yv - wright_omega<T>(z)) * T(kLog2e);
            }
          }
          A.G2[idx] = gn;
        }
      }
    }
    if (EPI == EPI_SOURCE) {
      // every lane of the warp holds the same problem p (or -1)
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (A.check && p >= 0 && lane == 0) atomicAdd(A.err_acc + p, part);
    }
  }
}

template <typename T>
struct MMArgs {
  const int* active;
  const int* n_active;
  int n, k;
  const T* D;       // [n][k]
  const T* Dt;      // [k][n]
  const T* xcol;    // [k] column sums of D
  const T* LA2;     // [P][n]
  T* S;             // [P][n] in: X w_prev, out: X w
  T* F2;            // [P][n] out: log2 S - LA2
  T* W;             // [P][k]
  T* mass;          // [P] sum_i S_i
  T* err_acc;       // [P] violation numerators (reset here)
  T* err;           // [P]
  T* dw;            // [P] ||w_new - w_old||_1 / ||w_new||_1 of the iteration's MM update
  const int* gap_ok;  // [P] relative duality gap <= gap_tol at this iteration's check
  int gap_check;    // this iteration evaluated the gap (gap_ok is current)
  int* done;
  int* iters;
  int* status;
  int it, max_iter;
  T tol, dw_tol;
  int gap_on;       // gap_tol > 0: the gap is a stopping criterion
  int penalty;
  int mm_steps = 1;  // MM steps with the same LA2 (a = K u1)
  T eps, alpha, beta;
};

// S = D w for problem p (rows strided over the block), F2 = log2 S - LA2 when LA2 != nullptr,
// and the mass sum_i S_i.
template <typename T>
__device__ __forceinline__ T source_marginal(const T* __restrict__ Dt, const T* w_s, int n, int k,
                                             T* __restrict__ S, T* __restrict__ F2, const T* __restrict__ LA2,
                                             T* red) {
  using P = Prec<T>;
  T mass = T(0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    T s = T(0);
    for (int j = 0; j < k; ++j) s = fma(Dt[(size_t)j * n + i], w_s[j], s);
    // a subnormal FP32 mass is taken as 0 (the log2 instruction flushes it to -inf); such a row
    // carries no source mass and drops out of the MM sum, as rows with s_i = 0 do
    if (s < P::tiny()) s = T(0);
    S[i] = s;
    if (F2) F2[i] = s > T(0) ? P::log2(s) - LA2[i] : P::ninf();
    mass += s;
  }
  return block_sum(mass, red);
}

// The stopping test of Algorithm 1's "while not converged" (reading A8): the source-marginal
// violation e <= tol, optionally together with the weight change ||dw||_1 / ||w||_1 <= dw_tol and a
// relative FP64 duality gap <= gap_tol (taken at check iterations only).  Every enabled criterion
// must hold; with none enabled the solve runs max_iter iterations.  Returns a status or -1.
// may_converge = false holds a problem back from a converged stop at this iteration (the tensor-core
// path while its applies still take the single BF16 product: a returned state always comes from
// hi/lo applies).
template <typename T>
__device__ __forceinline__ int stop_decision(T e, T dw, T tol, T dw_tol, bool gap_on, bool gap_ok, int it,
                                             int max_iter, bool may_converge = true) {
  if (e != e) return ST_NONFINITE;
  const bool any = tol > T(0) || dw_tol > T(0) || gap_on;
  if (may_converge && any && (!(tol > T(0)) || e <= tol) && (!(dw_tol > T(0)) || dw <= dw_tol) &&
      (!gap_on || gap_ok))
    return ST_CONVERGED;
  if (it >= max_iter) return ST_MAX_ITER;
  return -1;
}

// Per active problem (one CTA of 256 threads): convergence decision for the previous iteration,
// then Table 2's MM step  nu_j = log w_j + (ln2 / x_j) sum_i D_ij (LA2_i - log2 S_i)  (rows with
// S_i = 0 dropped), the penalty update and S = D w, mm_steps times with the same LA2; the last
// source step also writes F2 = log2 S - LA2.
template <typename T, int KQ>
__global__ void __launch_bounds__(256) mm_kernel(MMArgs<T> A) {
  using P = Prec<T>;
  constexpr int KP = KQ * 32;
  __shared__ T red_s[8][KP];
  __shared__ T w_s[KP];
  __shared__ T w0_s[KP];
  __shared__ T red[32];
  __shared__ int stop;
  const int slot = blockIdx.x;
  if (slot >= *A.n_active) return;
  const int p = A.active[slot];
  const int n = A.n, k = A.k;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* LA2 = A.LA2 + (size_t)p * n;
  T* S = A.S + (size_t)p * n;

  if (A.it > 0) {
    if (threadIdx.x == 0) {
      const T e = A.err_acc[p] / A.mass[p];
      A.err[p] = e;
      const int st = stop_decision<T>(e, A.dw[p], A.tol, A.dw_tol, A.gap_on != 0,
                                      A.gap_check && A.gap_ok && A.gap_ok[p], A.it, A.max_iter);
      if (st >= 0) {
        A.status[p] = st;
        A.iters[p] = A.it;
        A.done[p] = 1;
      }
      A.err_acc[p] = T(0);
      stop = st >= 0;
    }
    __syncthreads();
    if (stop) return;
  }

  for (int j = threadIdx.x; j < k; j += blockDim.x) w0_s[j] = A.W[(size_t)p * k + j];
  for (int m = 0; m < A.mm_steps; ++m) {
    // phase A: Dt r, r_i = LA2_i - log2 S_i (log2 units), 32 rows per warp step
    T acc[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) acc[q] = T(0);
    for (int base = warp * 32; base < n; base += 8 * 32) {
      const int i = base + lane;
      T r = T(0);
      if (i < n) {
        const T s = S[i];
        r = s > T(0) ? LA2[i] - P::log2(s) : T(0);
      }
      const int cnt = min(32, n - base);
      for (int t = 0; t < cnt; ++t) {
        const T rt = __shfl_sync(0xffffffffu, r, t);
        const T* Drow = A.D + (size_t)(base + t) * k;
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
          const int j = lane + 32 * q;
          if (j < k) acc[q] = fma(Drow[j], rt, acc[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < KQ; ++q) red_s[warp][lane + 32 * q] = acc[q];
    __syncthreads();

    // phase B: penalty update (Table 2)
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
      T sum = T(0);
#pragma unroll
      for (int w8 = 0; w8 < 8; ++w8) sum += red_s[w8][j];
      const T xj = A.xcol[j];
      const T wold = A.W[(size_t)p * k + j];
      const T nu = P::log(wold) + sum * T(kLn2) / xj;
      // l1 and elastic net: nu shifted by alpha/(eps x_j); squared l2 and elastic net:
      // W0(c e^nu)/c = omega(log c + nu)/c with c = alpha resp. beta over eps x_j (App. A)
      const T shift = (A.penalty == PEN_L1 || A.penalty == PEN_ELASTIC) ? A.alpha / (A.eps * xj) : T(0);
      T wn;
      if (A.penalty == PEN_L2SQ || A.penalty == PEN_ELASTIC) {
        const T c = (A.penalty == PEN_ELASTIC ? A.beta : A.alpha) / (A.eps * xj);
        wn = wright_omega<T>(P::log(c) + nu - shift) / c;
      } else wn = P::exp(nu - shift);
      A.W[(size_t)p * k + j] = wn;
      w_s[j] = wn;
    }
    __syncthreads();

    // phase C: source step
    const bool last = m + 1 == A.mm_steps;
    const T mass = source_marginal<T>(A.Dt, w_s, n, k, S, last ? A.F2 + (size_t)p * n : nullptr, LA2, red);
    if (last && threadIdx.x == 0) A.mass[p] = mass;
    __syncthreads();
  }
  // weight change of this iteration's update (all its MM steps): ||w - w_start||_1 / ||w||_1
  T num = T(0), den = T(0);
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    num += fabs(w_s[j] - w0_s[j]);
    den += fabs(w_s[j]);
  }
  num = block_sum(num, red);
  den = block_sum(den, red);
  if (threadIdx.x == 0) A.dw[p] = num / den;
}

// S = D w0 and its mass for every problem of the batch (one CTA per problem).
template <typename T>
__global__ void __launch_bounds__(256) source_init_kernel(const T* Dt, const T* W, T* S, T* mass, int n, int k) {
  __shared__ T w_s[256];
  __shared__ T red[32];
  const int p = blockIdx.x;
  for (int j = threadIdx.x; j < k; j += blockDim.x) w_s[j] = W[(size_t)p * k + j];
  __syncthreads();
  const T m = source_marginal<T>(Dt, w_s, n, k, S + (size_t)p * n, nullptr, nullptr, red);
  if (threadIdx.x == 0) mass[p] = m;
}

// Order-preserving removal of finished problems from the active list (one CTA, in place).
static __global__ void __launch_bounds__(1024) compact_kernel(int* active, int* n_active, const int* done) {
  __shared__ int warp_tot[32];
  __shared__ int total_s;
  const int na = *n_active;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int out = 0;
  for (int base = 0; base < na; base += 1024) {
    const int idx = base + threadIdx.x;
    const int p = idx < na ? active[idx] : -1;
    const int keep = (p >= 0 && !done[p]) ? 1 : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    const int before = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    if (warp == 0) {
      const int v = warp_tot[lane];
      int incl = v;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      warp_tot[lane] = incl - v;
      if (lane == 31) total_s = incl;
    }
    __syncthreads();
    if (keep) active[out + warp_tot[warp] + before] = p;
    out += total_s;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_active = out;
}

template <typename T>
struct PrepArgs {
  const T* x; const T* D; const T* w_in; const T* g_in; const T* y;
  T* xt; T* Dt; T* xcol; T* W; T* G2;
  int* active; int* done; int* n_active; T* err_acc; int* iters; int* status; T* err;
  T* dw; int* all; int* all_count;
  int batch, n, k;
  T xscale;    // 1 / sqrt(eps ln2)
  T gscale;    // 1 / (eps ln2)
};

// Per-solve preparation: scaled grid, transposed dictionary and its column sums, weights and
// potentials copied in, active list reset.  Grid-stride over the largest of the index spaces.
template <typename T>
__global__ void prep_kernel(PrepArgs<T> A) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nk = (size_t)A.n * A.k, bn = (size_t)A.batch * A.n, bk = (size_t)A.batch * A.k;
  if (A.x)  // NULL when the cost is given as a dense matrix
    if (A.x)  // no grid with a dense cost
      for (size_t e = tid; e < (size_t)A.n; e += stride) A.xt[e] = A.x[e] * A.xscale;
  for (size_t e = tid; e < nk; e += stride) {
    const size_t i = e / A.k, j = e - i * A.k;
    A.Dt[j * A.n + i] = A.D[e];
  }
  for (size_t e = tid; e < bk; e += stride) A.W[e] = A.w_in[e];
  for (size_t e = tid; e < bn; e += stride) A.G2[e] = A.g_in ? A.g_in[e] * A.gscale : T(0);
  for (size_t e = tid; e < (size_t)A.batch; e += stride) {
    A.active[e] = (int)e;
    A.done[e] = 0;
    A.err_acc[e] = T(0);
    A.iters[e] = 0;
    A.status[e] = ST_MAX_ITER;
    A.err[e] = T(0);
    A.dw[e] = Prec<T>::nan();
    A.all[e] = (int)e;
  }
  if (tid == 0) {
    *A.n_active = A.batch;
    *A.all_count = A.batch;
  }
}

// Column sums x_j of the dictionary (one warp per column).
template <typename T>
__global__ void colsum_kernel(const T* Dt, T* xcol, int n, int k) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= k) return;
  T s = T(0);
  for (int i = lane; i < n; i += 32) s += Dt[(size_t)j * n + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) xcol[j] = s;
}

template <typename T>
struct FinArgs {
  const T* W; const T* G2; const T* LB2; const int* iters; const int* status; const T* err;
  T* w_out; T* g_out; T* t_out; int* iters_out; int* status_out; T* err_out;
  int batch, n, k;
  T gscale_inv;  // eps ln2
};

// Copy the solver state out: w, g = eps ln2 G2, t = Q^T 1 = 2^(G2 + LB2), per-problem stats.
// Cold start of Algorithm 1 (reading A10: w0_j = sum(y) / (k x_j), x_j = sum_i D_ij; u1 = 1).
// cold_colsum_kernel: thread j sums column j of D [n][k] (FP64 accumulation; consecutive threads
// read consecutive atoms of a row); cold_weights_kernel: one CTA per problem.
template <typename T>
__global__ void cold_colsum_kernel(const T* D, int n, int k, T* xcol) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += (double)D[(size_t)i * k + j];
  xcol[j] = (T)s;
}
template <typename T>
__global__ void __launch_bounds__(256) cold_weights_kernel(const T* y, const T* xcol, int n, int k, T* w0) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)y[(size_t)b * n + i];
  s = block_sum(s, red);
  for (int j = threadIdx.x; j < k; j += blockDim.x) w0[(size_t)b * k + j] = (T)(s / ((double)k * (double)xcol[j]));
}

template <typename T>
__global__ void finalize_kernel(FinArgs<T> A) {
  using P = Prec<T>;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t bn = (size_t)A.batch * A.n, bk = (size_t)A.batch * A.k;
  for (size_t e = tid; e < bk; e += stride) A.w_out[e] = A.W[e];
  for (size_t e = tid; e < bn; e += stride) {
    if (A.g_out) A.g_out[e] = A.G2[e] * A.gscale_inv;
    if (A.t_out) A.t_out[e] = P::exp2(A.G2[e] + A.LB2[e]);
  }
  for (size_t e = tid; e < (size_t)A.batch; e += stride) {
    if (A.iters_out) A.iters_out[e] = A.iters[e];
    if (A.status_out) A.status_out[e] = A.status[e];
    if (A.err_out) A.err_out[e] = A.err[e];
  }
}

}  // namespace otlm
