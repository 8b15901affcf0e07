// Algorithm 1 for a banded cost and a sparse dictionary (the paper's scalability test: a cost
// truncated to C = +inf beyond a distance, so K_ij = 0 off a band of half-width h, and k = n/10
// truncated basis functions), FP32.
//
// The cost comes in diagonal storage Cd[d][i] = C(i, i + d - h), d = 0..2h (+inf: no pair).  With
// C2 = C / (eps ln2) the applies are
//   LA2_i = log2 sum_d 2^(G2_{i+d-h} - C2[d][i]),   LB2_j = log2 sum_e 2^(F2_{j+e-h} - C2[2h-e][j+e-h])
// (the target apply finds C(i, j), i = j + e - h, in diagonal 2h - e of row i).  K itself is never
// stored in HBM.  The dictionary is used in two sparse forms: the caller's CSC for D^T r (one
// thread per atom and problem) and a CSR copy built here for s = D w (one thread per row).
//
// One iteration is three launches: source apply (LA2, the violation numerator per tile, the log
// ratios r = LA2 - log2 S), MM step (stop decision from the tile partials in a fixed order, then
// Table 2 per atom and problem), and target kernel (s = D w on the tile and its halo, F2 =
// log2 s - LA2, the target apply and the datafit prox of Table 1, the tile's mass).  The apply
// kernels take tiles of 256 bins x PB (4) problems per CTA, three CTAs per SM: a thread owns one row (or column) of the
// band, loads its 2h + 1 costs once into registers (template buckets of 9, 19 and 33 diagonals,
// padded with +inf; wider bands read them from global memory) and uses them for the PB problems,
// whose potentials (tile plus halo) are staged in shared memory.  Each log-sum-exp is one pass of
// exp2 around the previous iteration's value of the same sum, which is also the ratio new / old
// the convergence test needs; a sum outside [2^-60, 2^60] is redone exactly (max, then sum).  A
// shared shift per window of rows would not do: at eps = 1e-3 the potentials move by ~14 log2
// units per bin, so a window's largest term underflows most of its rows' terms.
// A problem that stops keeps the state of its last completed iteration; later launches skip it.
//
// Precision of the potentials.  At eps = 1e-3 the log2 potentials reach lam / (eps ln2) ~ 1443, where
// an FP32 value resolves only ~6e-5 (a relative 4e-5 in u = 2^G), and the MM step's sum of
// D_ij log2(a_i / s_i) cancels terms of that size to a result near 0.  So G2, LA2 and LB2 are kept
// as pairs {a, b} (float2) whose value is a + b with `a` integer-valued (exact in FP32 up to 2^24)
// and |b| <= 1/2 after normalisation (pot_norm): the difference of two potentials' `a` parts is
// exact, and every rounding happens on numbers of the size of the result.  The datafit step and
// the MM sum take their few large-magnitude operations in FP64 (O(n) and O(nnz) per problem per
// iteration); the exponent-unit work stays FP32.
#pragma once

#include "banded_api.h"

namespace otlm {

constexpr int BAND_TN = 256;       // bins per tile (one per thread)
constexpr int BAND_NT = 256;       // threads per CTA

struct BandArgs {
  int batch, n, k, h, tiles, it, max_iter, datafit, penalty;
  float tol, eps, alpha, beta;
  // constants of the datafit step as FP32 pairs {hi, lo} (value hi + lo to ~48 bits): lam/(eps+lam),
  // lam/(eps ln2), lam/eps, ln(lam/eps), log2(eps/lam), ln 2
  float2 kl_coef, tv_bound, lam_over_eps, log_lam_over_eps, log2_eps_over_lam, ln2;
  const float* C2;        // [2h+1][n] C / (eps ln2)
  const int* col_ptr;     // [k+1]  CSC of D
  const int* row_idx;     // [nnz]
  const float* val;       // [nnz]
  const int* row_ptr;     // [n+1]  CSR copy of D
  const int* col_idx;     // [nnz]
  const float* rval;      // [nnz]
  const float* xcol;      // [k] column masses
  const float* y;         // [B][n]
  float2* G2;             // [B][n] target potential / (eps ln2), split {a, b}
  float2* LA2;            // [B][n] log2 K u1 (previous iteration's on entry to the source kernel), split
  float2* LB2;            // [B][n] log2 K^T u2 (previous iteration's on entry to the target kernel), split
  float* S;               // [B][n] D w
  float* W;               // [B][k]
  float* vpart;           // [B][tiles] violation numerators
  float* mpart;           // [B][tiles] masses sum_i S_i
  float* err;             // [B]
  int* done;
  int* iters;
  int* status;
  int* remaining;         // problems not yet stopped
};

constexpr int BAND_WARPS = BAND_NT / 32;

// Shared memory of the apply kernels (bytes): PB split potential rows [TN + 2h] (float2) and the
// block-sum scratch [PB][warps].
inline size_t band_smem_bytes(int h, int pb) {
  return 8 * (size_t)pb * (BAND_TN + 2 * (size_t)h) + 4 * (size_t)pb * BAND_WARPS;
}

// A split potential a + b with a integer-valued and |b| <= 1/2 (exact: rintf(b) and b - rintf(b)
// are representable, and a + rintf(b) stays an integer below 2^24).  -inf stays {-inf, 0}.
__device__ __forceinline__ float2 pot_norm(float a, float b) {
  const float r = rintf(b);
  return isfinite(a) ? make_float2(a + r, b - r) : make_float2(a, 0.f);
}
// The split of an FP64 value (the initial potentials).
__device__ __forceinline__ float2 pot_split(double v) {
  if (!isfinite(v)) return make_float2((float)v, 0.f);
  const double a = rint(v);
  return make_float2((float)a, (float)(v - a));
}
__device__ __forceinline__ double pot_value(float2 v) { return (double)v.x + (double)v.y; }

// Error-free transformations in FP32 (Dekker's product through the FMA, Knuth's two-sum): a b and
// a + b as exact pairs {value, rounding error}.  The intrinsics keep the compiler from fusing or
// reordering them.  They replace FP64, whose pipe is a small fraction of FP32's here.
__device__ __forceinline__ float2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return make_float2(p, __fmaf_rn(a, b, -p));
}
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
// A pair {hi, lo} (any |lo|) as a split potential.
__device__ __forceinline__ float2 pot_from_pair(float hi, float lo) {
  const float a = rintf(hi);
  return pot_norm(a, __fadd_rn(__fsub_rn(hi, a), lo));
}

// Staged split potentials of PB problems (PB even) in pair layout: column c of problems 2q and 2q+1
// is the float4 {a_2q, a_2q+1, b_2q, b_2q+1} at dst[q * L + c] (a: integer parts, b: fractions), so
// one 16-byte load feeds the packed (f32x2) arithmetic of both problems and a warp's load of 32
// consecutive columns is contiguous.
__device__ __forceinline__ float4 pair_put(float2 u, float2 v) { return make_float4(u.x, v.x, u.y, v.y); }
__device__ __forceinline__ float2 pair_get(const float4& q, int which) {
  return which ? make_float2(q.y, q.w) : make_float2(q.x, q.z);
}

// Stage PB split potential rows: problem p0 + pp, column c = src[p0 + pp][t0 - h + c] (-inf outside
// [0, n) or past the batch), in pair layout.
template <int PB>
__device__ __forceinline__ void band_stage_rows(const BandArgs& A, const float2* src, float4* dst, int p0, int t0,
                                                int L) {
  const float2 none = make_float2(-CUDART_INF_F, 0.f);
#pragma unroll
  for (int q = 0; q < PB / 2; ++q)
    for (int c = threadIdx.x; c < L; c += BAND_NT) {
      const int j = t0 - A.h + c;
      const bool in = j >= 0 && j < A.n;
      const int pa = p0 + 2 * q, pb = pa + 1;
      const float2 u = (in && pa < A.batch) ? src[(size_t)pa * A.n + j] : none;
      const float2 v = (in && pb < A.batch) ? src[(size_t)pb * A.n + j] : none;
      dst[q * L + c] = pair_put(u, v);
    }
}

// One row's band costs: WR > 0 keeps them in registers (cr, padded with +inf), otherwise they are
// read from global memory at cg[t * cgstride].
template <int WR>
struct BandRow {
  float cr[WR > 0 ? WR : 1];
  const float* cg;
  long cgstride;
  __device__ __forceinline__ float c(int t) const {
    if constexpr (WR > 0) return cr[t];
    else return cg[t * cgstride];
  }
};

// sum_t 2^(v_t - c_t - s) with split potentials, ((v_t.a - s.a) - c_t) + (v_t.b - s.b), where the
// first difference is exact and a term that matters has an exponent near 0 (so its rounding is
// relative to a small number), for the two problems of a pair at once (the pair at v, stride `st`
// float4 between columns): packed FP32 pairs (f32x2), two chains of additions in flight.
template <int WR>
__device__ __forceinline__ void band_sum2(const float4* v, int st, const BandRow<WR>& row, int T, float2 s0, float2 s1,
                                          float* sum0, float* sum1) {
  using P = Prec<float>;
  const uint64_t nsa = f2_pack(-s0.x, -s1.x), nsb = f2_pack(-s0.y, -s1.y);
  uint64_t acc0 = f2_pack(0.f, 0.f), acc1 = acc0;  // two chains of additions in flight
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const float4 q = v[t * st];
    const float nc = -row.c(t);
    const uint64_t e = f2_add(f2_add(f2_add(f2_pack(q.x, q.y), nsa), f2_pack(nc, nc)), f2_add(f2_pack(q.z, q.w), nsb));
    float e0, e1;
    f2_unpack(e, e0, e1);
    const uint64_t x = f2_pack(P::exp2(e0), P::exp2(e1));
    if (t & 1) acc1 = f2_add(acc1, x);
    else acc0 = f2_add(acc0, x);
  }
  f2_unpack(f2_add(acc0, acc1), *sum0, *sum1);
}

struct BandLse {
  float2 la;    // split log-sum
  float ratio;  // 2^(la - shift)
};
// The exact two passes for problem `which` of the pair at v (stride st): the largest term's exponent
// as the shift (a split value), then the sum around it; the band costs cg[t * cgstride], t < W.
// Out of line: rare, and it keeps the packed path's registers free.
__device__ __noinline__ BandLse band_lse_exact(const float4* v, int st, const float* cg, long cgstride, int W,
                                               int which, float2 sh) {
  using P = Prec<float>;
  float m = -CUDART_INF_F, ctm = 0.f;
  int tm = 0;
  for (int t = 0; t < W; ++t) {
    const float2 vt = pair_get(v[t * st], which);
    const float c = cg[t * cgstride];
    const float e = (vt.x - c) + vt.y;
    if (e > m) {
      m = e;
      tm = t;
      ctm = c;
    }
  }
  BandLse r;
  if (!(m > -CUDART_INF_F)) {
    r.la = make_float2(-CUDART_INF_F, 0.f);
    r.ratio = P::exp2(-CUDART_INF_F - sh.x);
    return r;
  }
  const float2 vm = pair_get(v[tm * st], which);
  const float2 s2 = pot_norm(vm.x, vm.y - ctm);
  float sa = 0.f, sb = 0.f;  // two chains, as the packed path
  for (int t = 0; t < W; ++t) {
    const float2 vt = pair_get(v[t * st], which);
    const float e = P::exp2(((vt.x - s2.x) - cg[t * cgstride]) + (vt.y - s2.y));
    if (t & 1) sb += e;
    else sa += e;
  }
  r.la = pot_norm(s2.x, s2.y + P::log2(sa + sb));
  r.ratio = P::exp2((r.la.x - sh.x) + (r.la.y - sh.y));
  return r;
}

// log2 sum_t 2^(v_t - c_t) over the row's band for the two problems of a pair: one pass around each
// problem's shift, the previous iteration's log-sum, so the sum is the ratio new / old; a problem
// whose shift is not finite or whose sum leaves [2^-60, 2^60] takes the exact two passes alone (the
// largest term as the shift, then the sum around it).  Returns the split log-sums and the ratios
// 2^(new - shift).
template <int WR>
__device__ __forceinline__ void band_lse2(const float4* v, int st, const BandRow<WR>& row, int W, float2 sh0,
                                          float2 sh1, float2* la0, float2* la1, float* ratio0, float* ratio1) {
  using P = Prec<float>;
  constexpr bool REG = WR > 0;
  const int T = REG ? WR : W;
  float sum0 = 0.f, sum1 = 0.f;
  const bool f0 = isfinite(sh0.x), f1 = isfinite(sh1.x);
  if (f0 || f1)
    band_sum2<WR>(v, st, row, T, f0 ? sh0 : make_float2(0.f, 0.f), f1 ? sh1 : make_float2(0.f, 0.f), &sum0, &sum1);
  const bool ok0 = f0 && sum0 >= 0x1p-60f && sum0 <= 0x1p60f, ok1 = f1 && sum1 >= 0x1p-60f && sum1 <= 0x1p60f;
  if (ok0) {
    *ratio0 = sum0;
    *la0 = pot_norm(sh0.x, sh0.y + P::log2(sum0));
  }
  if (ok1) {
    *ratio1 = sum1;
    *la1 = pot_norm(sh1.x, sh1.y + P::log2(sum1));
  }
  if (!ok0 || !ok1) {  // rare: the exact path, one problem at a time, with the band read from memory
    if (!ok0) {
      const BandLse r = band_lse_exact(v, st, row.cg, row.cgstride, W, 0, sh0);
      *la0 = r.la;
      *ratio0 = r.ratio;
    }
    if (!ok1) {
      const BandLse r = band_lse_exact(v, st, row.cg, row.cgstride, W, 1, sh1);
      *la1 = r.la;
      *ratio1 = r.ratio;
    }
  }
}

// Fixed-order block sum of PB per-thread values; thread pp < PB gets the total of value pp.
template <int PB>
__device__ __forceinline__ float band_block_sums(const float (&v)[PB], float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int pp = 0; pp < PB; ++pp) {
    float x = v[pp];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[pp * BAND_WARPS + warp] = x;
  }
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x < PB)
    for (int w8 = 0; w8 < BAND_WARPS; ++w8) t += red[threadIdx.x * BAND_WARPS + w8];
  return t;
}

template <int PB>
__device__ __forceinline__ bool band_live(const BandArgs& A, int p0, bool (&live)[PB]) {
  bool any = false;
#pragma unroll
  for (int pp = 0; pp < PB; ++pp) {
    live[pp] = p0 + pp < A.batch && !A.done[p0 + pp];
    any |= live[pp];
  }
  return any;
}

__device__ __forceinline__ bool band_live_one(const BandArgs& A, int p) { return p < A.batch && !A.done[p]; }

// Sum of a problem's tile partials in a fixed order (lane-strided, then a fixed shuffle tree).
__device__ __forceinline__ float band_tile_sum(const float* part, int tiles) {
  const int lane = threadIdx.x & 31;
  float v = 0.f;
  for (int t = lane; t < tiles; t += 32) v += part[t];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Source apply for PB problems on one tile of rows: LA2 and the violation numerator
// sum_i S_i |a_new,i / a_old,i - 1|.  Row i's costs C2[d][i] are loaded once (coalesced across the
// tile) for the PB problems.
template <int PB, int WR>
__global__ void __launch_bounds__(BAND_NT, 3) band_source_kernel(BandArgs A) {
  extern __shared__ __align__(16) float smem[];
  const int tile = blockIdx.x, p0 = blockIdx.y * PB;
  const int n = A.n, h = A.h, W = 2 * h + 1, L = BAND_TN + 2 * h, t0 = tile * BAND_TN;
  bool live[PB];
  if (!band_live<PB>(A, p0, live)) return;
  static_assert(PB % 2 == 0, "problems go in pairs");
  float4* gs = reinterpret_cast<float4*>(smem);
  float* red = smem + 2 * (size_t)PB * L;
  band_stage_rows<PB>(A, A.G2, gs, p0, t0, L);
  const int i = t0 + threadIdx.x;
  const bool valid = i < n;
  BandRow<WR> row;
  row.cg = A.C2 + (valid ? i : 0);
  row.cgstride = n;
  if constexpr (WR > 0) {
#pragma unroll
    for (int t = 0; t < WR; ++t) row.cr[t] = (valid && t < W) ? A.C2[(size_t)t * n + i] : CUDART_INF_F;
  }
  // the PB problems' previous sums and masses of row i, loaded before any is used
  float2 old[PB];
  float sv[PB];
#pragma unroll
  for (int pp = 0; pp < PB; ++pp) {
    const size_t o = (size_t)(p0 + pp) * n + i;
    old[pp] = (live[pp] && valid) ? A.LA2[o] : make_float2(0.f, 0.f);
    sv[pp] = (live[pp] && valid) ? A.S[o] : 0.f;
  }
  __syncthreads();
  const bool check = A.it > 0;
  float part[PB];
#pragma unroll
  for (int q = 0; q < PB / 2; ++q) {
    const int pa = 2 * q, pb = pa + 1;
    part[pa] = part[pb] = 0.f;
    if (!valid || !(live[pa] || live[pb])) continue;
    float2 la[2];
    float ratio[2];
    band_lse2<WR>(gs + q * L + threadIdx.x, 1, row, W, old[pa], old[pb], &la[0], &la[1], &ratio[0], &ratio[1]);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int pp = pa + u;
      if (!live[pp]) continue;
      if (check && sv[pp] > 0.f) part[pp] = sv[pp] * fabsf(ratio[u] - 1.f);
      A.LA2[(size_t)(p0 + pp) * n + i] = la[u];
    }
  }
  if (!check) return;
  const float tot = band_block_sums<PB>(part, red);
  if (threadIdx.x < PB && band_live_one(A, p0 + threadIdx.x))
    A.vpart[(size_t)(p0 + threadIdx.x) * A.tiles + tile] = tot;
}

// One problem (blockIdx.y) x 256 atoms per CTA: warp 0 takes the problem's stop decision from the
// tile partials (every CTA of the problem reaches the same one; the first records it), then each
// thread runs Table 2's MM step for its atom.
__global__ void __launch_bounds__(BAND_NT) band_mm_kernel(BandArgs A) {
  using P = Prec<float>;
  __shared__ int stop_s;
  const int p = blockIdx.y;
  if (A.done[p]) return;
  if (A.it > 0) {
    if (threadIdx.x < 32) {
      const float num = band_tile_sum(A.vpart + (size_t)p * A.tiles, A.tiles);
      const float mass = band_tile_sum(A.mpart + (size_t)p * A.tiles, A.tiles);
      if (threadIdx.x == 0) {
        const float e = num / mass;
        int st = -1;
        if (e != e) st = ST_NONFINITE;
        else if (A.tol > 0.f && e <= A.tol) st = ST_CONVERGED;
        else if (A.it >= A.max_iter) st = ST_MAX_ITER;
        if (blockIdx.x == 0) {
          A.err[p] = e;
          if (st >= 0) {
            A.status[p] = st;
            A.iters[p] = A.it;
            A.done[p] = 1;
            atomicSub(A.remaining, 1);
          }
        }
        stop_s = st >= 0;
      }
    }
    __syncthreads();
    if (stop_s) return;
  }
  const int m = blockIdx.x * BAND_NT + threadIdx.x;
  if (m >= A.k) return;
  // sum_i D_im log2(a_i / s_i) with log2(a / s) = la.a + (la.b - log2 s): the integer parts are of
  // size up to lam / (eps ln2) and the weighted sum cancels to near 0 at the fixed point, so their
  // products and running sum are kept exact as FP32 pairs (two_prod, two_sum)
  const float2* LA = A.LA2 + (size_t)p * A.n;
  const float* S = A.S + (size_t)p * A.n;
  const int q0 = A.col_ptr[m], q1 = A.col_ptr[m + 1];
  float hi = 0.f, lo = 0.f;
  auto add = [&](float v, int r) {
    const float sv = S[r];
    if (!(sv > 0.f)) return;
    const float2 la = LA[r];
    const float2 pr = two_prod(v, la.x);
    const float2 sm = two_sum(hi, pr.x);
    hi = sm.x;
    lo += (sm.y + pr.y) + v * (la.y - P::log2(sv));
  };
  int q = q0;
  for (; q + 4 <= q1; q += 4) {  // four independent gathers in flight
    const int r0 = A.row_idx[q], r1 = A.row_idx[q + 1], r2 = A.row_idx[q + 2], r3 = A.row_idx[q + 3];
    const float v0 = A.val[q], v1 = A.val[q + 1], v2 = A.val[q + 2], v3 = A.val[q + 3];
    add(v0, r0);
    add(v1, r1);
    add(v2, r2);
    add(v3, r3);
  }
  for (; q < q1; ++q) add(A.val[q], A.row_idx[q]);
  const float xj = A.xcol[m];
  float* wp = A.W + (size_t)p * A.k + m;
  const float nu = P::log(*wp) + (hi + lo) * float(kLn2) / xj;
  const float shift = (A.penalty == PEN_L1 || A.penalty == PEN_ELASTIC) ? A.alpha / (A.eps * xj) : 0.f;
  float wn;
  if (A.penalty == PEN_L2SQ || A.penalty == PEN_ELASTIC) {
    const float c = (A.penalty == PEN_ELASTIC ? A.beta : A.alpha) / (A.eps * xj);
    wn = wright_omega<float>(P::log(c) + nu - shift) / c;
  } else wn = P::exp(nu - shift);
  *wp = wn;
}

// log2 omega(z) for z = zh + zl (a pair): omega of zh, corrected to first order for zl
// (omega' = omega / (1 + omega)), so |z| ~ 1e3 costs no FP32 resolution.
__device__ __forceinline__ float log2_omega(float zh, float zl) {
  using P = Prec<float>;
  const float om = wright_omega_fast(zh);
  return P::log2(om) + zl * float(kLog2e) * P::rcp(1.f + om);
}

// c_hi x + (c_lo x) for an integer-valued x and a constant pair c: exact up to the last term.
__device__ __forceinline__ float2 pair_times(float2 c, float x) {
  float2 p = two_prod(c.x, x);
  p.y = __fmaf_rn(c.y, x, p.y);
  return p;
}

// Datafit step (Table 1) in log2 units from the split target sum v = log2 b and the target bin y,
// as a split potential.  The large parts (v's integer part, lam y / eps, the TV bound, the KL
// factor) are combined through exact FP32 pairs; the squared-error and Poisson steps use their log
// forms
//   L2     : G2 = log2(eps/lam) + log2 omega(ln(lam/eps) + v ln2 + (lam/eps) y) - v,
//   Poisson: G2 = l2c - log2 omega((l2c - v) ln2 + lam/eps) - v, l2c = log2(lam y / eps)
// (no difference of two numbers of size lam y / eps, which the FP32 form lam y/eps - omega had).
__device__ __noinline__ float2 band_datafit(const BandArgs& A, float2 v, float yv) {
  using P = Prec<float>;
  const float ly = P::log2(yv);
  switch (A.datafit) {
    case DF_BALANCED: return pot_norm(-v.x, ly - v.y);
    case DF_KL: {  // kl (ly - v.b) - kl v.a
      const float2 pa = pair_times(A.kl_coef, -v.x);
      const float2 pb = two_prod(A.kl_coef.x, ly);
      const float2 sm = two_sum(pa.x, pb.x);
      return pot_from_pair(sm.x, sm.y + pa.y + pb.y + A.kl_coef.y * ly - A.kl_coef.x * v.y);
    }
    case DF_TV: {
      const float2 g = pot_norm(-v.x, ly - v.y);
      // compare g with the bound pair: (g.a - bound.hi) is exact near the bound
      const float over = (g.x - A.tv_bound.x) + (g.y - A.tv_bound.y);
      const float under = (g.x + A.tv_bound.x) + (g.y + A.tv_bound.y);
      if (over > 0.f) return pot_from_pair(A.tv_bound.x, A.tv_bound.y);
      if (under < 0.f) return pot_from_pair(-A.tv_bound.x, -A.tv_bound.y);
      return g;
    }
    case DF_POISSON: {  // reading A7; -lam where y = 0
      if (!(yv > 0.f)) return pot_from_pair(-A.tv_bound.x, -A.tv_bound.y);
      // l2c = log2(lam/eps) + ly; z = ln2 (l2c - v.b) - ln2 v.a + lam/eps
      const float l2c = ly - A.log2_eps_over_lam.x;
      const float2 za = pair_times(A.ln2, -v.x);
      const float2 zb = two_prod(A.ln2.x, l2c - v.y);
      const float2 s1 = two_sum(za.x, A.lam_over_eps.x);
      const float2 s2 = two_sum(s1.x, zb.x);
      const float zl = s1.y + s2.y + za.y + zb.y + A.lam_over_eps.y - A.ln2.x * A.log2_eps_over_lam.y;
      const float2 z = two_sum(s2.x, zl);
      const float lo = log2_omega(z.x, z.y);
      return pot_norm(-v.x, (l2c - lo) - v.y - A.log2_eps_over_lam.y);
    }
    default: {  // L2: z = ln(lam/eps) + ln2 v.a + ln2 v.b + (lam/eps) y
      const float2 za = pair_times(A.ln2, v.x);
      const float2 zy = two_prod(A.lam_over_eps.x, yv);
      const float2 s1 = two_sum(za.x, zy.x);
      const float2 s2 = two_sum(s1.x, A.log_lam_over_eps.x);
      const float zl = s1.y + s2.y + za.y + zy.y + A.lam_over_eps.y * yv + A.log_lam_over_eps.y + A.ln2.x * v.y;
      const float2 z = two_sum(s2.x, zl);
      const float lo = log2_omega(z.x, z.y);
      return pot_norm(-v.x, ((A.log2_eps_over_lam.x + lo) - v.y) + A.log2_eps_over_lam.y);
    }
  }
}

// Source step, target apply and datafit prox for PB problems on one tile: s = D w over the tile and
// its halo (CSR rows, shared by the PB problems), F2 = log2 s - LA2, then LB2 and G2 (Table 1).
// Column j's costs C(j + e - h, j) = C2[2h - e][j + e - h] are loaded once for the PB problems.
template <int PB, int WR>
__global__ void __launch_bounds__(BAND_NT, 3) band_target_kernel(BandArgs A) {
  using P = Prec<float>;
  extern __shared__ __align__(16) float smem[];
  const int tile = blockIdx.x, p0 = blockIdx.y * PB;
  const int n = A.n, h = A.h, W = 2 * h + 1, L = BAND_TN + 2 * h, t0 = tile * BAND_TN;
  bool live[PB];
  if (!band_live<PB>(A, p0, live)) return;
  static_assert(PB % 2 == 0, "problems go in pairs");
  float4* fs = reinterpret_cast<float4*>(smem);
  float* red = smem + 2 * (size_t)PB * L;
  float mass[PB];
#pragma unroll
  for (int pp = 0; pp < PB; ++pp) mass[pp] = 0.f;
  for (int c = threadIdx.x; c < L; c += BAND_NT) {
    const int i = t0 - h + c;
    float s[PB];
#pragma unroll
    for (int pp = 0; pp < PB; ++pp) s[pp] = 0.f;
    if (i >= 0 && i < n) {
      const int e0 = A.row_ptr[i], e1 = A.row_ptr[i + 1];
      for (int e = e0; e < e1; ++e) {
        const size_t col = (size_t)A.col_idx[e];
        const float v = A.rval[e];
#pragma unroll
        for (int pp = 0; pp < PB; ++pp)
          if (live[pp]) s[pp] = fmaf(v, A.W[(size_t)(p0 + pp) * A.k + col], s[pp]);
      }
    }
    const bool own = c >= h && c < h + BAND_TN && i < n;
    float2 f2s[PB];
#pragma unroll
    for (int pp = 0; pp < PB; ++pp) {
      float2 f2 = make_float2(-CUDART_INF_F, 0.f);
      if (live[pp] && i >= 0 && i < n) {
        // a subnormal mass counts as 0, as in the other FP32 paths (log2 flushes it to -inf)
        const float sv = s[pp] < P::tiny() ? 0.f : s[pp];
        const size_t o = (size_t)(p0 + pp) * n + i;
        if (sv > 0.f) {
          const float2 la = A.LA2[o];
          f2 = pot_norm(-la.x, P::log2(sv) - la.y);  // F2 = log2 s - LA2
        }
        if (own) {
          A.S[o] = sv;
          mass[pp] += sv;
        }
      }
      f2s[pp] = f2;
    }
#pragma unroll
    for (int q = 0; q < PB / 2; ++q) fs[q * L + c] = pair_put(f2s[2 * q], f2s[2 * q + 1]);
  }
  const int j = t0 + threadIdx.x;
  const bool valid = j < n;
  // term e of column j: row j + e - h, diagonal 2h - e, i.e. C2 + (2h - e) n + j + e - h
  BandRow<WR> col;
  col.cg = A.C2 + (valid ? (long)(2 * h) * n + j - h : 0);
  col.cgstride = 1 - (long)n;
  if constexpr (WR > 0) {
#pragma unroll
    for (int t = 0; t < WR; ++t) {
      const int i = j + t - h;
      col.cr[t] = (valid && t < W && i >= 0 && i < n) ? A.C2[(size_t)(2 * h - t) * n + i] : CUDART_INF_F;
    }
  }
  // the PB problems' previous sums and targets of column j, loaded before any is used
  float2 old[PB];
  float yv[PB];
#pragma unroll
  for (int pp = 0; pp < PB; ++pp) {
    const size_t o = (size_t)(p0 + pp) * n + j;
    old[pp] = (live[pp] && valid) ? A.LB2[o] : make_float2(0.f, 0.f);
    yv[pp] = (live[pp] && valid) ? A.y[o] : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PB / 2; ++q) {
    const int pa = 2 * q, pb = pa + 1;
    if (!valid || !(live[pa] || live[pb])) continue;
    float2 lb[2];
    float ratio[2];
    band_lse2<WR>(fs + q * L + threadIdx.x, 1, col, W, old[pa], old[pb], &lb[0], &lb[1], &ratio[0], &ratio[1]);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int pp = pa + u;
      if (!live[pp]) continue;
      const size_t o = (size_t)(p0 + pp) * n + j;
      A.LB2[o] = lb[u];
      A.G2[o] = band_datafit(A, lb[u], yv[pp]);
    }
  }
  const float tot = band_block_sums<PB>(mass, red);
  if (threadIdx.x < PB && band_live_one(A, p0 + threadIdx.x))
    A.mpart[(size_t)(p0 + threadIdx.x) * A.tiles + tile] = tot;
}

// ---- set-up: scaled cost band, CSR copy of the dictionary, column masses, initial state -------

// C2[d][i] = Cd[d][i] / (eps ln2); any NaN or -inf entry flags the input as invalid.
__global__ void band_cost_kernel(const float* Cd, float* C2, size_t count, float inv, int* bad) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < count; q += (size_t)gridDim.x * blockDim.x) {
    const float c = Cd[q];
    if (c != c || c == -CUDART_INF_F) atomicOr(bad, 1);
    C2[q] = c * inv;
  }
}

// Per atom: the column's entries must lie in [0, n) with non-negative values, its pointers must
// be ordered and its mass positive; counts entries per row.
__global__ void band_csc_check_kernel(const int* col_ptr, const int* row_idx, const float* val, int n, int k,
                                      int nnz, float* xcol, int* cnt, int* bad) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > k) return;
  if (m == k) {
    if (col_ptr[0] != 0 || col_ptr[k] != nnz) atomicOr(bad, 1);
    return;
  }
  const int a = col_ptr[m], b = col_ptr[m + 1];
  if (a < 0 || b < a || b > nnz) {
    atomicOr(bad, 1);
    return;
  }
  float s = 0.f;
  for (int q = a; q < b; ++q) {
    const int r = row_idx[q];
    const float v = val[q];
    if (r < 0 || r >= n || !(v >= 0.f)) {
      atomicOr(bad, 1);
      continue;
    }
    atomicAdd(cnt + r, 1);
    s += v;
  }
  xcol[m] = s;
  if (!(s > 0.f)) atomicOr(bad, 1);
}

// Exclusive scan of the row counts into row_ptr [n+1] (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) band_scan_kernel(const int* cnt, int* row_ptr, int n) {
  __shared__ int warp_tot[32];
  __shared__ int carry_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < n ? cnt[i] : 0;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const int wv = warp_tot[lane];
      int wi = wv;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      warp_tot[lane] = wi - wv;
    }
    __syncthreads();
    const int carry = carry_s;
    if (i < n) row_ptr[i] = carry + warp_tot[warp] + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry_s = carry + warp_tot[31] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) row_ptr[n] = carry_s;
}

// Scatter the CSC entries into their rows (positions by atomics), then sort every row by atom
// index so that the row sums of s = D w run in a fixed order.
__global__ void band_fill_kernel(const int* col_ptr, const int* row_idx, const float* val, int k, const int* row_ptr,
                                 int* fill, int* col_idx, float* rval) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= k) return;
  for (int q = col_ptr[m]; q < col_ptr[m + 1]; ++q) {
    const int r = row_idx[q];
    const int pos = row_ptr[r] + atomicAdd(fill + r, 1);
    col_idx[pos] = m;
    rval[pos] = val[q];
  }
}

__global__ void band_sort_rows_kernel(const int* row_ptr, int* col_idx, float* rval, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = row_ptr[i], b = row_ptr[i + 1];
  for (int q = a + 1; q < b; ++q) {  // insertion sort by (atom, value): rows hold a few entries
    const int c = col_idx[q];
    const float v = rval[q];
    int t = q - 1;
    while (t >= a && (col_idx[t] > c || (col_idx[t] == c && rval[t] > v))) {
      col_idx[t + 1] = col_idx[t];
      rval[t + 1] = rval[t];
      --t;
    }
    col_idx[t + 1] = c;
    rval[t + 1] = v;
  }
}

// Initial state per problem: W = w0, G2 = g0 / (eps ln2) (0 for a cold start), S = D w0 (CSR rows),
// status MAX_ITER, not done.  One thread per (problem, row) for G2 and S, per (problem, atom) for W.
__global__ void band_init_kernel(BandArgs A, const float* w0, const float* g0, double gscale) {
  const size_t rows = (size_t)A.batch * A.n, atoms = (size_t)A.batch * A.k;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < atoms; q += (size_t)gridDim.x * blockDim.x)
    A.W[q] = w0[q];
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < rows; q += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(q / A.n), i = (int)(q - (size_t)p * A.n);
    A.G2[q] = g0 ? pot_split((double)g0[q] * gscale) : make_float2(0.f, 0.f);
    float s = 0.f;
    for (int e = A.row_ptr[i]; e < A.row_ptr[i + 1]; ++e) s = fmaf(A.rval[e], w0[(size_t)p * A.k + A.col_idx[e]], s);
    A.S[q] = s < Prec<float>::tiny() ? 0.f : s;
    A.LA2[q] = make_float2(-CUDART_INF_F, 0.f);  // no previous sums: the first applies take the exact path
    A.LB2[q] = make_float2(-CUDART_INF_F, 0.f);
  }
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < (size_t)A.batch;
       q += (size_t)gridDim.x * blockDim.x) {
    A.done[q] = 0;
    A.iters[q] = 0;
    A.status[q] = ST_MAX_ITER;
    A.err[q] = CUDART_NAN_F;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.remaining = A.batch;
}

// Outputs: w, g = G2 eps ln2, t = Q^T 1 = 2^(G2 + LB2) (0 before the first target step), iters,
// err, status.
__global__ void band_finalize_kernel(BandArgs A, float* w_out, float* g_out, float* t_out, int* iters_out,
                                     float* err_out, int* status_out, double gscale_inv) {
  const size_t rows = (size_t)A.batch * A.n, atoms = (size_t)A.batch * A.k;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < atoms; q += (size_t)gridDim.x * blockDim.x)
    w_out[q] = A.W[q];
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < rows; q += (size_t)gridDim.x * blockDim.x) {
    const float2 g = A.G2[q];
    if (g_out) g_out[q] = (float)(pot_value(g) * gscale_inv);
    if (t_out) {
      const float2 lb = A.LB2[q];  // t = 2^(G2 + LB2): integer parts added exactly
      t_out[q] = lb.x > -CUDART_INF_F ? Prec<float>::exp2((g.x + lb.x) + (g.y + lb.y)) : 0.f;
    }
  }
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < (size_t)A.batch;
       q += (size_t)gridDim.x * blockDim.x) {
    if (iters_out) iters_out[q] = A.iters[q];
    if (err_out) err_out[q] = A.err[q];
    if (status_out) status_out[q] = A.status[q];
  }
}

// Device workspace of the banded path (allocated by the handle on first use and grown on demand).
struct BandWorkspace {
  float* C2;
  int *row_ptr, *cnt, *fill, *col_idx;
  float *rval, *xcol;
  float2 *G2, *LA2, *LB2;
  float *S, *W, *vpart, *mpart, *err;
  int *done, *iters, *status, *remaining, *bad;
};

inline size_t carve_band_workspace(void* base, int batch, int n, int k, int h, int nnz, BandWorkspace* ws) {
  size_t off = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* p = b ? b + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  const size_t W = 2 * (size_t)h + 1, rows = (size_t)batch * n;
  const size_t tiles = (size_t)(n + BAND_TN - 1) / BAND_TN;
  BandWorkspace w;
  w.C2 = (float*)take(4 * W * n);
  w.row_ptr = (int*)take(4 * ((size_t)n + 1));
  w.cnt = (int*)take(4 * (size_t)n);
  w.fill = (int*)take(4 * (size_t)n);
  w.col_idx = (int*)take(4 * (size_t)nnz);
  w.rval = (float*)take(4 * (size_t)nnz);
  w.xcol = (float*)take(4 * (size_t)k);
  w.G2 = (float2*)take(8 * rows);
  w.LA2 = (float2*)take(8 * rows);
  w.LB2 = (float2*)take(8 * rows);
  w.S = (float*)take(4 * rows);
  w.W = (float*)take(4 * (size_t)batch * k);
  w.vpart = (float*)take(4 * (size_t)batch * tiles);
  w.mpart = (float*)take(4 * (size_t)batch * tiles);
  w.err = (float*)take(4 * (size_t)batch);
  w.done = (int*)take(4 * (size_t)batch);
  w.iters = (int*)take(4 * (size_t)batch);
  w.status = (int*)take(4 * (size_t)batch);
  w.remaining = (int*)take(4);
  w.bad = (int*)take(4);
  if (ws) *ws = w;
  return off;
}

// The iteration loop with PB problems per apply CTA and register-held bands of WR diagonals (0:
// read from global memory); polls the number of unfinished problems every poll_every iterations.
template <int PB, int WR>
cudaError_t band_iterate(const Launch& L, BandArgs& A, const BandWorkspace& ws, const SolveParams& sp) {
  const size_t smem = band_smem_bytes(A.h, PB);
  const dim3 grid_rows(A.tiles, (A.batch + PB - 1) / PB), grid_atoms((A.k + BAND_NT - 1) / BAND_NT, A.batch);
  for (int it = 0;; ++it) {
    A.it = it;
    L.begin(KIND_APPLY);
    band_source_kernel<PB, WR><<<grid_rows, BAND_NT, smem, L.stream>>>(A);
    L.end();
    L.begin(KIND_MM);
    band_mm_kernel<<<grid_atoms, BAND_NT, 0, L.stream>>>(A);
    L.end();
    if (it >= sp.max_iter) break;
    L.begin(KIND_APPLY);
    band_target_kernel<PB, WR><<<grid_rows, BAND_NT, smem, L.stream>>>(A);
    L.end();
    if ((it + 1) % sp.poll_every == 0) {
      cudaError_t e = cudaMemcpyAsync(L.host_flag, ws.remaining, sizeof(int), cudaMemcpyDeviceToHost, L.stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
      if (e == cudaSuccess && L.timer && L.timer->on) e = L.timer->harvest();
      if (e != cudaSuccess) return e;
      if (*L.host_flag == 0) break;
    }
  }
  return cudaGetLastError();
}

// Dispatch on problems per CTA (4 for batches of 4 or more, else 1) and the band-width bucket (9,
// 19 or 33 diagonals in registers, padded with +inf; wider bands from global memory).
template <int PB>
cudaError_t band_iterate_pb(const Launch& L, BandArgs& A, const BandWorkspace& ws, const SolveParams& sp) {
  const int W = 2 * A.h + 1;
  if (W <= 9) return band_iterate<PB, 9>(L, A, ws, sp);
  if (W <= 19) return band_iterate<PB, 19>(L, A, ws, sp);
  if (W <= 33) return band_iterate<PB, 33>(L, A, ws, sp);
  return band_iterate<PB, 0>(L, A, ws, sp);
}

// Returns the first CUDA error; *invalid is set when the band or the dictionary is malformed
// (checked on the device before any index from them is used).
inline cudaError_t solve_device_band(const Launch& L, const BandWorkspace& ws, const SolveParams& sp,
                                     const BandCall& c, bool* invalid) {
  *invalid = false;
  const int n = c.n, k = c.k, h = c.h, W = 2 * h + 1;
  const double eps_ln2 = sp.eps * kLn2;
  BandArgs A{};
  A.batch = c.batch; A.n = n; A.k = k; A.h = h; A.tiles = (n + BAND_TN - 1) / BAND_TN;
  A.max_iter = sp.max_iter; A.datafit = sp.datafit; A.penalty = sp.penalty;
  A.tol = float(sp.tol); A.eps = float(sp.eps); A.alpha = float(sp.alpha); A.beta = float(sp.beta);
  auto pair = [](double v) { const float h = (float)v; return make_float2(h, (float)(v - (double)h)); };
  A.kl_coef = pair(sp.lam / (sp.eps + sp.lam)); A.tv_bound = pair(sp.lam / eps_ln2);
  A.lam_over_eps = pair(sp.lam / sp.eps); A.log_lam_over_eps = pair(log(sp.lam / sp.eps));
  A.log2_eps_over_lam = pair(log2(sp.eps / sp.lam)); A.ln2 = pair(kLn2);
  A.C2 = ws.C2; A.col_ptr = c.col_ptr; A.row_idx = c.row_idx; A.val = c.val;
  A.row_ptr = ws.row_ptr; A.col_idx = ws.col_idx; A.rval = ws.rval; A.xcol = ws.xcol; A.y = c.y;
  A.G2 = ws.G2; A.LA2 = ws.LA2; A.LB2 = ws.LB2; A.S = ws.S; A.W = ws.W;
  A.vpart = ws.vpart; A.mpart = ws.mpart; A.err = ws.err; A.done = ws.done; A.iters = ws.iters;
  A.status = ws.status; A.remaining = ws.remaining;

  cudaError_t e = cudaMemsetAsync(ws.cnt, 0, sizeof(int) * n, L.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws.fill, 0, sizeof(int) * n, L.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws.bad, 0, sizeof(int), L.stream);
  if (e != cudaSuccess) return e;
  L.begin(KIND_OTHER);
  band_cost_kernel<<<592, 256, 0, L.stream>>>(c.Cd, ws.C2, (size_t)W * n, float(1.0 / eps_ln2), ws.bad);
  L.end();
  L.begin(KIND_OTHER);
  band_csc_check_kernel<<<(k + 1 + 255) / 256, 256, 0, L.stream>>>(c.col_ptr, c.row_idx, c.val, n, k, c.nnz,
                                                                   ws.xcol, ws.cnt, ws.bad);
  L.end();
  e = cudaMemcpyAsync(L.host_flag, ws.bad, sizeof(int), cudaMemcpyDeviceToHost, L.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
  if (e != cudaSuccess) return e;
  if (*L.host_flag) {
    *invalid = true;
    return cudaSuccess;
  }
  L.begin(KIND_OTHER);
  band_scan_kernel<<<1, 1024, 0, L.stream>>>(ws.cnt, ws.row_ptr, n);
  L.end();
  L.begin(KIND_OTHER);
  band_fill_kernel<<<(k + 255) / 256, 256, 0, L.stream>>>(c.col_ptr, c.row_idx, c.val, k, ws.row_ptr, ws.fill,
                                                          ws.col_idx, ws.rval);
  L.end();
  L.begin(KIND_OTHER);
  band_sort_rows_kernel<<<(n + 255) / 256, 256, 0, L.stream>>>(ws.row_ptr, ws.col_idx, ws.rval, n);
  L.end();
  L.begin(KIND_OTHER);
  band_init_kernel<<<1184, 256, 0, L.stream>>>(A, c.w, c.g, 1.0 / eps_ln2);
  L.end();

  e = c.batch >= 4 ? band_iterate_pb<4>(L, A, ws, sp) : band_iterate_pb<2>(L, A, ws, sp);
  if (e != cudaSuccess) return e;
  L.begin(KIND_OTHER);
  band_finalize_kernel<<<1184, 256, 0, L.stream>>>(A, c.w, c.g, c.t_out, c.iters_out, c.err_out, c.status_out,
                                                   eps_ln2);
  L.end();
  e = cudaGetLastError();
  if (e == cudaSuccess && L.timer && L.timer->on) e = L.timer->harvest();
  return e;
}

}  // namespace otlm
