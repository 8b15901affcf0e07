// Uneven batch in one persistent launch: every problem has its own grid x [n_p], dictionary
// D [n_p][k_p], eps_p and target y [n_p] (concatenated, with offsets).  One CTA solves one problem
// at a time, all of its iterations (Algorithm 1), with the problem's state in shared memory:
//   xt (scaled grid), G2, LA2, F2, LB2, S  (6 n_p floats) and W, xcol, reduction scratch.
// CTAs take problems from a device-side queue (an atomic counter over an order sorted by
// decreasing n_p^2, i.e. largest work first), so the 256x spread in work per problem balances
// across the SMs without any host round trip.
//
// The kernel apply inside a CTA: thread t owns R consecutive rows (R even, a compile-time
// constant picked from n_p); with its own centre c_t (the middle of its rows) the exponent
// in_j - m_i - (xt_i - xt_j)^2 becomes FFMA(2 di, dj, h_j) - q_i with h_j = in_j - dj^2 formed
// once per column and q_i = m_i + di^2 once per row; rows are processed in packed pairs
// (fma/add.f32x2).  Shift: the previous sums (later iterations), the diagonal term (first
// iteration), or an exact max pass when any sum leaves [2^-60, 2^60].
#pragma once

#include "kernels.cuh"

namespace otlm {

struct RaggedArgs {
  int batch;
  const int* order;   // problem ids, largest work first
  int* next;          // queue position (zeroed before the launch)
  const int* n;
  const int* k;
  const float* eps;
  const long long* off_n;  // start of problem p in x, y, g, t
  const long long* off_D;  // start of problem p in D
  const long long* off_k;  // start of problem p in w
  const float* x;
  const float* D;
  const float* y;
  float* w;                // in: initial weights (> 0), out: result
  const float* g_in;       // initial target potentials (eps log u1) or null
  float* g_out;            // final potentials or null
  float* t_out;            // transported target marginal or null
  int* iters;
  float* err;
  int* status;
  int datafit, penalty, max_iter;
  float lam, alpha, tol;
  float beta;                     // squared-l2 weight of the elastic net
  int mm_steps;                   // MM steps per iteration (>= 1)
  int n_max, k_max;
  long long tot_n, tot_D, tot_k;  // packed sizes of x/y, D and w (sum n, sum n k, sum k)
  int smem_floats;                // dynamic shared memory of the launch, in floats
  // rows per thread by size bucket (n in (256 b, 256 (b + 1)]), as log2 R; raised to the fewest
  // that cover n with this CTA size (0: always the fewest)
  unsigned char rows_log2[16];
};

constexpr int RAGGED_BUCKETS = 16;
__host__ __device__ inline int ragged_bucket(int n) { return n <= 256 ? 0 : (n - 1) / 256 < 15 ? (n - 1) / 256 : 15; }

template <int NT>
struct RaggedSmem {
  // offsets (floats) into dynamic shared memory for a problem of n_max bins, k_max atoms
  static __host__ __device__ size_t floats(int n_max, int k_max) {
    return 6 * (size_t)n_max + 2 * (size_t)k_max + (NT / 32) * (size_t)k_max + 64;
  }
};

// Sum pass of the in-CTA apply: acc2 = sum_j 2^(FFMA(2 di, dj, h_j) + nq) on packed row pairs.
template <int R>
__device__ __forceinline__ void ragged_sum(const float* xt, const float* in, int n, int i0, float xc,
                                           const uint64_t (&nq2)[R / 2], uint64_t (&acc2)[R / 2]) {
  using P = Prec<float>;
  constexpr int QP = R / 2;
  uint64_t tdi2[QP];
#pragma unroll
  for (int q = 0; q < QP; ++q) {
    const int a = min(i0 + 2 * q, n - 1), b = min(i0 + 2 * q + 1, n - 1);
    tdi2[q] = f2_pack(2.f * (xt[a] - xc), 2.f * (xt[b] - xc));
    acc2[q] = f2_pack(0.f, 0.f);
  }
#pragma unroll 2
  for (int j = 0; j < n; ++j) {
    const float dj = xt[j] - xc;
    const float h = fmaf(-dj, dj, in[j]);
    const uint64_t dj2 = f2_pack(dj, dj), h2 = f2_pack(h, h);
#pragma unroll
    for (int q = 0; q < QP; ++q) {
      const uint64_t u2 = f2_add(f2_fma(tdi2[q], dj2, h2), nq2[q]);
      float u0, u1;
      f2_unpack(u2, u0, u1);
      acc2[q] = f2_add(acc2[q], f2_pack(P::exp2(u0), P::exp2(u1)));
    }
  }
}

// One kernel apply inside the CTA: out_i = log2 sum_j 2^(in_j - (xt_i - xt_j)^2) for i < n.
// shift_prev: out holds the previous sums (shift = out_i); otherwise the diagonal in_i.
// ratio (optional): ratio_i = a_new_i / a_old_i (exact when the previous-sum shift held).
// Rows past n are computed on clamped rows and never stored.  Live through the column loop:
// three packed registers per row pair (shift, offset, accumulator).
template <int NT, int R>
__device__ void ragged_apply(const float* xt, const float* in, float* out, int n, bool shift_prev, float* ratio) {
  using P = Prec<float>;
  constexpr int QP = R / 2;
  const int i0 = threadIdx.x * R;
  const bool active = i0 < n;
  const float xc = active ? 0.5f * (xt[i0] + xt[min(i0 + R - 1, n - 1)]) : 0.f;
  const float* src = shift_prev ? out : in;
  bool bad = false;
  uint64_t nq2[QP], acc2[QP];
#pragma unroll
  for (int q = 0; q < QP; ++q) {
    float v[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = min(i0 + 2 * q + c, n - 1);
      const float m = active ? src[i] : 0.f;
      const float d = active ? xt[i] - xc : 0.f;
      bad |= active && !isfinite(m);
      v[c] = -(m + d * d);
    }
    nq2[q] = f2_pack(v[0], v[1]);
  }
  bool exact = __syncthreads_or(bad);
  if (!exact) {
    if (active) ragged_sum<R>(xt, in, n, i0, xc, nq2, acc2);
    bool b2 = false;
#pragma unroll
    for (int q = 0; q < QP; ++q) {
      float a0, a1;
      f2_unpack(acc2[q], a0, a1);
      b2 |= active && !(a0 >= 8.673617379884035e-19f && a0 <= 1.152921504606847e18f);
      b2 |= active && !(a1 >= 8.673617379884035e-19f && a1 <= 1.152921504606847e18f);
    }
    exact = __syncthreads_or(b2);
  }
  if (exact) {
    // exact shift: m_i = max_j (in_j - (xt_i - xt_j)^2), then the sum again
    float m[R];
#pragma unroll
    for (int r = 0; r < R; ++r) m[r] = -CUDART_INF_F;
    if (active)
      for (int j = 0; j < n; ++j) {
        const float dj = xt[j] - xc;
        const float h = fmaf(-dj, dj, in[j]);
#pragma unroll
        for (int r = 0; r < R; ++r) m[r] = fmaxf(m[r], fmaf(2.f * (xt[min(i0 + r, n - 1)] - xc), dj, h));
      }
#pragma unroll
    for (int q = 0; q < QP; ++q) {
      float v[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int r = 2 * q + c;
        const float d = active ? xt[min(i0 + r, n - 1)] - xc : 0.f;
        float mm = m[r] - d * d;
        if (!(mm > -CUDART_INF_F)) mm = 0.f;  // every term vanishes
        v[c] = -(mm + d * d);
      }
      nq2[q] = f2_pack(v[0], v[1]);
    }
    if (active) ragged_sum<R>(xt, in, n, i0, xc, nq2, acc2);
  }
  __syncthreads();  // every thread has read `out` and `in` before `out` is overwritten
  const bool prev_ratio = shift_prev && !exact;
#pragma unroll
  for (int q = 0; q < QP; ++q) {
    float nq[2], acc[2];
    f2_unpack(nq2[q], nq[0], nq[1]);
    f2_unpack(acc2[q], acc[0], acc[1]);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = i0 + 2 * q + c;
      if (!active || i >= n) continue;
      const float d = xt[i] - xc;
      const float v = acc[c] > 0.f ? (-nq[c] - d * d) + P::log2(acc[c]) : P::ninf();
      if (ratio) ratio[i] = prev_ratio ? acc[c] : (shift_prev ? P::exp2(v - out[i]) : 1.f);
      out[i] = v;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ float block_sum_f(float v, float* red) { return block_sum<float>(v, red); }

template <int NT, int R>
__device__ void ragged_solve_one(const RaggedArgs& A, int p, float* sm) {
  using P = Prec<float>;
  const int n = A.n[p], k = A.k[p];
  const float eps = A.eps[p];
  const float eps_ln2 = eps * float(kLn2);
  const long long on = A.off_n[p], oD = A.off_D[p], ok = A.off_k[p];
  // a problem whose sizes or offsets fall outside the packed arrays is marked invalid and not
  // touched; the barrier also separates the previous problem's last reads from this one's writes
  const bool valid = n >= 2 && n <= A.n_max && k >= 1 && k <= A.k_max && (n + NT - 1) / NT <= R && on >= 0 &&
                     on + n <= A.tot_n && oD >= 0 && oD + (long long)n * k <= A.tot_D && ok >= 0 &&
                     ok + k <= A.tot_k &&
                     6 * (long long)A.n_max + 2 * A.k_max + (NT / 32) * A.k_max + 64 <= A.smem_floats;
  if (!__syncthreads_and(valid)) {
    if (threadIdx.x == 0) {
      A.iters[p] = 0;
      A.err[p] = CUDART_NAN_F;
      A.status[p] = ST_INVALID;
    }
    return;
  }
  const float* D = A.D + oD;
  float* xt = sm;
  float* G2 = xt + A.n_max;
  float* LA2 = G2 + A.n_max;
  float* F2 = LA2 + A.n_max;
  float* LB2 = F2 + A.n_max;
  float* S = LB2 + A.n_max;
  float* W = S + A.n_max;
  float* xcol = W + A.k_max;
  float* red_k = xcol + A.k_max;  // [NT/32][k_max]
  float* red = red_k + (NT / 32) * A.k_max;  // 32 floats + scalars
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;

  const float xs = rsqrtf(eps_ln2);
  for (int i = tid; i < n; i += NT) {
    xt[i] = A.x[on + i] * xs;
    G2[i] = A.g_in ? A.g_in[on + i] / eps_ln2 : 0.f;
  }
  for (int j = tid; j < k; j += NT) W[j] = A.w[ok + j];
  // column sums x_j: warps over rows, lanes over columns
  for (int j0 = 0; j0 < k; j0 += 32) {
    float part = 0.f;
    const int j = j0 + lane;
    if (j < k)
      for (int i = warp; i < n; i += NW) part += D[(size_t)i * k + j];
    if (j < k) red_k[warp * A.k_max + j] = part;
  }
  __syncthreads();
  for (int j = tid; j < k; j += NT) {
    float s = 0.f;
    for (int w8 = 0; w8 < NW; ++w8) s += red_k[w8 * A.k_max + j];
    xcol[j] = s;
  }
  __syncthreads();

  // S = D w (warp per row, lanes over atoms), mass
  auto source_step = [&](bool write_f2) -> float {
    float mass = 0.f;
    for (int i = warp; i < n; i += NW) {
      float s = 0.f;
      for (int j = lane; j < k; j += 32) s = fmaf(D[(size_t)i * k + j], W[j], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (s < P::tiny()) s = 0.f;
      if (lane == 0) {
        S[i] = s;
        if (write_f2) F2[i] = s > 0.f ? P::log2(s) - LA2[i] : P::ninf();
      }
      mass += s;  // identical in every lane
    }
    __syncthreads();
    float tot = lane == 0 ? mass : 0.f;
    return block_sum_f(tot, red);
  };
  float mass = source_step(false);

  int it = 0;
  float e = 0.f;
  int st = ST_MAX_ITER;
  for (;; ++it) {
    // source apply; F2 doubles as the ratio buffer a_new / a_old
    ragged_apply<NT, R>(xt, G2, LA2, n, it > 0, F2);
    if (it > 0) {
      float part = 0.f;
      for (int i = tid; i < n; i += NT)
        if (S[i] > 0.f) part += S[i] * fabsf(F2[i] - 1.f);
      part = block_sum_f(part, red);
      e = part / mass;
      if (e != e) { st = ST_NONFINITE; break; }
      if (A.tol > 0.f && e <= A.tol) { st = ST_CONVERGED; break; }
    }
    if (it >= A.max_iter) { st = ST_MAX_ITER; break; }
    // MM step: nu_j = log w_j + (ln2 / x_j) sum_i D_ij (LA2_i - log2 S_i), then S = D w; mm_steps
    // times with the same LA2, the last one also writing F2
    for (int m = 0; m < A.mm_steps; ++m) {
      for (int j0 = 0; j0 < k; j0 += 32) {
        const int j = j0 + lane;
        float part = 0.f;
        if (j < k)
          for (int i = warp; i < n; i += NW) {
            const float s = S[i];
            if (s > 0.f) part = fmaf(D[(size_t)i * k + j], LA2[i] - P::log2(s), part);
          }
        if (j < k) red_k[warp * A.k_max + j] = part;
      }
      __syncthreads();
      for (int j = tid; j < k; j += NT) {
        float sum = 0.f;
        for (int w8 = 0; w8 < NW; ++w8) sum += red_k[w8 * A.k_max + j];
        const float xj = xcol[j];
        const float nu = P::log(W[j]) + sum * float(kLn2) / xj;
        const float shift = (A.penalty == PEN_L1 || A.penalty == PEN_ELASTIC) ? A.alpha / (eps * xj) : 0.f;
        float wn;
        if (A.penalty == PEN_L2SQ || A.penalty == PEN_ELASTIC) {
          const float c = (A.penalty == PEN_ELASTIC ? A.beta : A.alpha) / (eps * xj);
          wn = wright_omega<float>(P::log(c) + nu - shift) / c;
        } else wn = P::exp(nu - shift);
        W[j] = wn;
      }
      __syncthreads();
      const float m_mass = source_step(m + 1 == A.mm_steps);
      if (m + 1 == A.mm_steps) mass = m_mass;
    }
    // target apply and the datafit step (Table 1) in log2 units
    ragged_apply<NT, R>(xt, F2, LB2, n, it > 0, nullptr);
    const float kl_coef = A.lam / (eps + A.lam), tv_bound = A.lam / eps_ln2, loe = A.lam / eps;
    const float lloe = logf(A.lam / eps);
    for (int j = tid; j < n; j += NT) {
      const float v = LB2[j], yv = A.y[on + j];
      float gn;
      switch (A.datafit) {
        case DF_BALANCED: gn = P::log2(yv) - v; break;
        case DF_KL: gn = kl_coef * (P::log2(yv) - v); break;
        case DF_TV: gn = fminf(fmaxf(P::log2(yv) - v, -tv_bound), tv_bound); break;
        default: {  // L2 or Poisson (reading A7; -lam where y = 0), one Wright omega
          const bool pois = A.datafit == DF_POISSON;
          if (pois && !(yv > 0.f)) {
            gn = -tv_bound;
            break;
          }
          const float l2c = pois ? lloe * float(kLog2e) + P::log2(yv) : 0.f;
          const float z = pois ? (l2c - v) * float(kLn2) + loe : lloe + v * float(kLn2) + loe * yv;
          const float om = wright_omega<float>(z);
          gn = pois ? l2c - P::log2(om) - v : (loe * yv - om) * float(kLog2e);
        }
      }
      G2[j] = gn;
    }
    __syncthreads();
  }
  // outputs
  for (int j = tid; j < k; j += NT) A.w[ok + j] = W[j];
  for (int i = tid; i < n; i += NT) {
    if (A.g_out) A.g_out[on + i] = G2[i] * eps_ln2;
    if (A.t_out) A.t_out[on + i] = it > 0 ? P::exp2(G2[i] + LB2[i]) : 0.f;
  }
  if (tid == 0) {
    A.iters[p] = it;
    A.err[p] = e;
    A.status[p] = st;
  }
  __syncthreads();
}

// Persistent kernel: CTAs take problems from the queue until it is empty.  RMAX = rows per
// thread for the largest n the handle supports (n_max <= NT * RMAX).
template <int NT, int RMAX>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) ragged_kernel(RaggedArgs A) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_idx;
  for (;;) {
    if (threadIdx.x == 0) s_idx = atomicAdd(A.next, 1);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= A.batch) break;
    const int p = A.order[idx];
    const int n = A.n[p];
    // rows per thread: the tuned choice for n's size bucket, at least the fewest that cover n
    // (more rows per thread amortise each column's shared-memory reads over more exponentials,
    // fewer keep more threads busy)
    const int need = (n + NT - 1) / NT;
    int rows = 1 << (A.rows_log2[ragged_bucket(n)] > 0 ? A.rows_log2[ragged_bucket(n)] : 1);
    while (rows < need) rows <<= 1;
    if (rows <= 2) ragged_solve_one<NT, 2>(A, p, sm);
    else if (RMAX >= 4 && rows <= 4) ragged_solve_one<NT, (RMAX >= 4 ? 4 : 2)>(A, p, sm);
    else if (RMAX >= 8 && rows <= 8) ragged_solve_one<NT, (RMAX >= 8 ? 8 : 2)>(A, p, sm);
    else if (RMAX >= 16 && rows <= 16) ragged_solve_one<NT, (RMAX >= 16 ? 16 : 2)>(A, p, sm);
    else if (RMAX >= 32 && rows <= 32) ragged_solve_one<NT, (RMAX >= 32 ? 32 : 2)>(A, p, sm);
    else if (threadIdx.x == 0) {  // more rows per thread than this CTA size supports
      A.iters[p] = 0;
      A.err[p] = CUDART_NAN_F;
      A.status[p] = ST_INVALID;
    }
  }
}

}  // namespace otlm

namespace otlm {

// Variants the tuner chooses among: CTA size NT with rows per thread up to RMAX (n <= 4096).
constexpr int RAGGED_VARIANTS = 3;
inline int ragged_nt(int v) { return v == 0 ? 128 : (v == 1 ? 256 : 512); }
inline int ragged_rmax_log2(int v) { return v == 0 ? 5 : (v == 1 ? 4 : 3); }

inline cudaError_t ragged_prepare(int v, int n_max, int k_max, int* blocks_per_sm, size_t* smem) {
  const int nt = ragged_nt(v);
  size_t bytes = 0;
  const void* fn = nullptr;
  if (v == 0) { bytes = RaggedSmem<128>::floats(n_max, k_max) * 4; fn = (const void*)ragged_kernel<128, 32>; }
  else if (v == 1) { bytes = RaggedSmem<256>::floats(n_max, k_max) * 4; fn = (const void*)ragged_kernel<256, 16>; }
  else { bytes = RaggedSmem<512>::floats(n_max, k_max) * 4; fn = (const void*)ragged_kernel<512, 8>; }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, nt, bytes);
  *smem = bytes;
  return e;
}

inline void ragged_launch(int v, dim3 grid, size_t smem, cudaStream_t s, const RaggedArgs& a) {
  if (v == 0) ragged_kernel<128, 32><<<grid, 128, smem, s>>>(a);
  else if (v == 1) ragged_kernel<256, 16><<<grid, 256, smem, s>>>(a);
  else ragged_kernel<512, 8><<<grid, 512, smem, s>>>(a);
}

}  // namespace otlm
