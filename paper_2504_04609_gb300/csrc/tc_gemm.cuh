// tcgen05 (5th-generation tensor core) three-term GEMM, sm_100a/sm_103a.
//
//   out[map(c)][r] = sum_j ( Ahi[r][j] Bhi[c][j] + Ahi[r][j] Blo[c][j] + Alo[r][j] Bhi[c][j] )
//
// (or, on request through a device flag read at launch, the single product Ahi Bhi^T: one MMA per
// k step on the hi tiles alone; the solver uses it while every problem is far from convergence)
//
// Both operands are K-major (contiguous along j) and carried as hi/lo pairs (x = hi + lo), so the
// three products recover most of the precision the single-pass type drops:
//   KIND_BF16 (kind::f16, BF16 operands): ~16 mantissa bits; the kernel applies K V^T, where A = the
//             Gibbs kernel K (rows r = grid bins) and B = the scaled scalings of the batch;
//   KIND_TF32 (kind::tf32, FP32 containers rounded to TF32): ~21 bits; the dictionary contractions
//             D w (A = D, B = the weights) and D^T r (A = D^T, B = the log ratios).
// Accumulation is FP32 in tensor memory (TMEM); the epilogue stores FP32 sums, optionally through a
// column map, with an optional split of the reduction (each split stores its own partial sums,
// added later in a fixed order).
//
// Two kernels: gemm3_pair_kernel (below; SM pairs, cta_group::2) for every GEMM whose reduction is
// not split (the applies of larger batches, D w), and gemm3_kernel for split reductions (small batches,
// D^T r) and the warm-start network.  gemm3_kernel is a persistent
// kernel, one CTA per SM; work units (128 x 128 output tile, reduction split) are dealt round-robin
// over the CTAs:
//   warp 0 lane 0: TMA producer (cp.async.bulk.tensor, 128B-swizzled tiles, a 192 KiB ring that runs
//                  on across units: 3 stages of the four hi/lo tiles, or 6 stages of the two hi
//                  tiles when the single product is requested, so that twice as many k blocks are
//                  in flight while each one feeds a third of the tensor work)
//   warp 1 lane 0: MMA issuer  (3 x 4 tcgen05.mma per 128-byte k block) into one of two TMEM
//                  accumulators, so the epilogue of unit i overlaps the MMAs of unit i + 1
//   warps 4..7   : epilogue    (tcgen05.ld 32x32b, one TMEM lane quarter per warp; 64 columns at a
//                  time, four loads per wait, through a 32 KiB staging buffer and one bulk copy per
//                  output column, or stored from registers on request)
// Every wait on an mbarrier is bounded (about 2 s of %globaltimer, or GemmArgs.wait_ns); on expiry
// the CTA records an error in *err, stops issuing work, lets its issued copies land, waits boundedly
// for its committed MMAs and frees its TMEM.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace otlm {
namespace tc {

enum { KIND_BF16 = 0, KIND_TF32 = 1 };
constexpr int BM = 128, BN = 128, BK_BYTES = 128, STAGES = 3;
constexpr int A_TILE = BM * BK_BYTES;                     // 16 KiB
constexpr int B_TILE = BN * BK_BYTES;                     // 16 KiB
constexpr int STAGE_BYTES = 2 * A_TILE + 2 * B_TILE;      // 64 KiB: A hi, B hi, A lo, B lo
constexpr int STAGES_SINGLE = STAGE_BYTES * STAGES / (A_TILE + B_TILE);  // 6 stages of A hi, B hi
constexpr int EPI_BYTES = 64 * BM * 4;                    // 32 KiB: 64 output columns of 128 rows
constexpr int NBARS = 2 * STAGES_SINGLE + 5;              // full[6], empty[6], acc_full[2], acc_empty[2], drain
constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + EPI_BYTES + NBARS * 8 + 16;
constexpr int THREADS = 256;
constexpr uint32_t TMEM_COLS = 2 * BN;                    // two accumulators (double buffer)
// Sums below 2^-90 (relative to the operand's shift) are listed for an exact recomputation: their
// terms' BF16 lo parts (2^-9 below the hi parts) and hi x lo products approach FP32's subnormal
// range, where they flush to zero; above 2^-90 every term that matters keeps all its bits.
constexpr float EXACT_BELOW = 8.0779356694631609e-28f;    // 2^-90
static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");
constexpr unsigned long long WAIT_NS = 2000000000ull;    // bounded waits: 2 s

enum { ERR_NONE = 0, ERR_WAIT_TMA = 1, ERR_WAIT_MMA = 2, ERR_WAIT_ACC = 3 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of the barrier; false after `lim` ns.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long lim = WAIT_NS) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > lim) return false;
  return true;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}
// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row atoms 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);  // start address (16-byte units)
  d |= static_cast<uint64_t>(1) << 16;                  // leading-dimension offset (unused with this swizzle)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;          // stride between 8-row atoms
  d |= static_cast<uint64_t>(1) << 46;                  // descriptor version (fixed 0b001)
  d |= static_cast<uint64_t>(2) << 61;                  // 128-byte swizzle
  return d;
}
// Elements per 128-byte k block and per MMA (each MMA consumes 32 bytes of k).
template <int KIND> struct KindTraits;
template <> struct KindTraits<KIND_BF16> { static constexpr int BK = 64, FMT = 1; };  // BF16
template <> struct KindTraits<KIND_TF32> { static constexpr int BK = 32, FMT = 2; };  // TF32

// Instruction descriptor: FP32 accumulator, A and B of the same format (BF16 = 1 under kind::f16,
// TF32 = 2 under kind::tf32), both K-major, M x N.
template <int KIND>
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (static_cast<uint32_t>(KindTraits<KIND>::FMT) << 7) |
         (static_cast<uint32_t>(KindTraits<KIND>::FMT) << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}
template <int KIND>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t id,
                                     uint32_t accumulate) {
  if constexpr (KIND == KIND_BF16)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(id), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(id), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }


// tcgen05.ld of 16 columns without the wait: several loads in flight, then one tmem_wait_ld.
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// Wait for the loads issued so far; the 64 destination registers pass through the waits so that no
// use of them is scheduled before the loads have landed.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[64]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 64; j += 16)
    asm volatile(""
                 : "+r"(v[j]), "+r"(v[j + 1]), "+r"(v[j + 2]), "+r"(v[j + 3]), "+r"(v[j + 4]), "+r"(v[j + 5]),
                   "+r"(v[j + 6]), "+r"(v[j + 7]), "+r"(v[j + 8]), "+r"(v[j + 9]), "+r"(v[j + 10]), "+r"(v[j + 11]),
                   "+r"(v[j + 12]), "+r"(v[j + 13]), "+r"(v[j + 14]), "+r"(v[j + 15])::"memory");
}

struct GemmArgs {
  float* out;          // out[z * split_stride + map(c) * ld_out + r]
  const int* col_map;  // column (slot) -> output row; nullptr: identity
  const int* n_cols;   // number of valid columns on the device; nullptr: N
  int M, N, Kd, ld_out;
  int* err;            // first error code of any CTA (0: none)
  int2* fix_list;                // sums below EXACT_BELOW as (output row, row); nullptr: not recorded
  unsigned long long* fix_cnt;   // entries this launch appended to fix_list
  unsigned long long fix_cap;    // capacity of fix_list (M x N covers every element)
  int flush_tiny;      // store sums below FLT_MIN as 0
  int splits;          // the reduction is split into `splits` ranges of k blocks; >= 1
  size_t split_stride; // elements between the partial-sum planes of consecutive splits
  int bulk;            // set by launch_gemm3: every output column segment is 16-byte aligned and a
                       // multiple of 16 bytes long, so the tile leaves through shared memory as
                       // one bulk copy per column
  const int* hilo;     // null: the three products; otherwise, while *hilo == 0 (read at launch),
                       // the single product hi x hi: only the hi tiles are loaded
  int store_direct;    // 1: the epilogue stores from registers, one 128-byte segment per warp and
                       // column, instead of staging and one bulk copy per column
  unsigned long long wait_ns;  // limit of every barrier wait (0: WAIT_NS)
  int withhold;        // self-check of the expired-wait path (otlm_check_wait_expiry): the producer of
                       // the first CTA arms its first stage but never issues the copies, so the MMA
                       // issuer's wait on that stage runs out; 0 in every solve
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Named barrier 1 over the four epilogue warps with an OR of `v`: every warp gets the same answer.
__device__ __forceinline__ bool bar_or_epi(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(v))
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void bulk_store(float* gdst, uint32_t ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(ssrc), "r"(bytes)
               : "memory");
}

// Epilogue of one 128 x BN output tile in TMEM (the calling warp's lane quarter q: rows
// m0 + 32 q + lane; columns n0 .. n0 + BN - 1 at TMEM column offsets tq + c), 64 columns at a time:
// four loads and one wait per half, then either the 32 KiB staging buffer and one bulk copy per
// column (g.bulk) or one 128-byte store per warp and column. release() runs once every TMEM read of
// the tile is done. Sums below EXACT_BELOW are listed for the exact fix-up.
template <class Release>
__device__ __forceinline__ void epilogue_tile(const GemmArgs& g, float* out, uint32_t tq, float* stage_out,
                                              uint32_t stage_s, int m0, int n0, int ncols, int q, int lane, int et,
                                              Release release) {
  const int row = m0 + q * 32 + lane;
  const int ncol_tile = min(BN, ncols - n0);
  const int rows = min(BM, g.M - m0);  // <= 0: the tile's rows all lie past the last row
  for (int h = 0; h < BN / 64; ++h) {
    if (g.bulk) {
      if (et < 64) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // staging is free again
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
    // the half's 64 columns (columns past the last problem are read too: the buffer holds all BN)
    uint32_t v[64];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 4; ++j) tmem_ld16_nowait(tq + static_cast<uint32_t>(h * 64 + j * 16), v + 16 * j);
    tmem_wait_ld(v);
    if (h == BN / 64 - 1) {
      tc_fence_before();
      __syncwarp();
      release();
    }
    // direct stores: the output rows of the half's 64 columns, two per lane, read once
    int orow0 = 0, orow1 = 0;
    if (!g.bulk) {
      const int c0 = n0 + h * 64 + lane, c1 = c0 + 32;
      orow0 = c0 < ncols ? (g.col_map ? g.col_map[c0] : c0) : 0;
      orow1 = c1 < ncols ? (g.col_map ? g.col_map[c1] : c1) : 0;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c0 = h * 64 + j * 16;
      unsigned low = 0;  // columns whose sum is below EXACT_BELOW (including an empty sum)
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int col = n0 + c0 + c;
        const bool in = col < ncols && row < g.M;
        float val = __uint_as_float(v[16 * j + c]);
        low |= (in && !(val >= EXACT_BELOW)) ? (1u << c) : 0u;
        if (g.flush_tiny && val < 1.17549435e-38f) val = 0.f;  // a NaN stays visible
        if (g.bulk) {
          stage_out[(c0 - h * 64 + c) * BM + q * 32 + lane] = val;
        } else {  // one 128-byte segment per warp and column
          const int cc = j * 16 + c;  // column within the half (compile-time)
          const int o = __shfl_sync(0xffffffffu, cc < 32 ? orow0 : orow1, cc & 31);
          if (in) out[static_cast<size_t>(o) * g.ld_out + row] = val;
        }
      }
      if (low && g.fix_list) {  // rare: list each underflowed sum for the exact fix-up
        for (; low; low &= low - 1) {
          const int col = n0 + c0 + __ffs(low) - 1;
          const unsigned long long e = atomicAdd(g.fix_cnt, 1ull);
          if (e < g.fix_cap) g.fix_list[e] = make_int2(g.col_map ? g.col_map[col] : col, row);
        }
      }
    }
    if (g.bulk) {
      // the generic-proxy writes become visible to the bulk-copy (async) proxy, then one thread per
      // column sends rows m0 .. m0 + rows - 1 of that column
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("bar.sync 1, 128;" ::: "memory");
      const int c = h * 64 + et;
      if (et < 64 && c < ncol_tile && rows > 0) {
        const int o = g.col_map ? g.col_map[n0 + c] : n0 + c;
        bulk_store(out + static_cast<size_t>(o) * g.ld_out + m0, stage_s + static_cast<uint32_t>(et) * (BM * 4),
                   static_cast<uint32_t>(rows) * 4u);
      }
      if (et < 64) asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
}

template <int KIND>
__global__ void __launch_bounds__(THREADS, 1)
    gemm3_kernel(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
                 const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo, GemmArgs g) {
  constexpr int BK = KindTraits<KIND>::BK;
  extern __shared__ uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncols = g.n_cols ? *g.n_cols : g.N;
  const bool three = !g.hilo || *g.hilo != 0;  // the three products, or hi x hi alone
  const int nst = three ? STAGES : STAGES_SINGLE;  // ring stages of this launch
  const unsigned long long lim = g.wait_ns ? g.wait_ns : WAIT_NS;
  const uint32_t st_bytes = three ? STAGE_BYTES : A_TILE + B_TILE;
  const int mt = (g.M + BM - 1) / BM, nt = (g.N + BN - 1) / BN;
  const int units = mt * nt * g.splits;
  const int nkb_all = (g.Kd + BK - 1) / BK;
  // work unit u -> output tile (m0, n0) and reduction split z (m fastest)
  auto coords = [&](int u, int* m0, int* n0, int* z) {
    *m0 = (u % mt) * BM;
    const int r = u / mt;
    *n0 = (r % nt) * BN;
    *z = r / nt;
  };
  // split z's k blocks (the host keeps splits <= blocks, so every split has at least one)
  auto krange = [&](int z, int* kb0, int* nkb) {
    *kb0 = static_cast<int>(static_cast<long long>(nkb_all) * z / g.splits);
    *nkb = static_cast<int>(static_cast<long long>(nkb_all) * (z + 1) / g.splits) - *kb0;
  };

  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* const stage_out = reinterpret_cast<float*>(base + STAGES * STAGE_BYTES);  // [64 columns][128 rows]
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES + EPI_BYTES);
  // full[STAGES_SINGLE], empty[STAGES_SINGLE], acc_full[2], acc_empty[2], drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NBARS);
  int* fail = reinterpret_cast<int*>(tmem_slot + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES_SINGLE);
  const uint32_t accf0 = smem_u32(bars + 2 * STAGES_SINGLE), acce0 = smem_u32(bars + 2 * STAGES_SINGLE + 2);
  const uint32_t drain = smem_u32(bars + 2 * STAGES_SINGLE + 4);
  const uint32_t ring = smem_u32(base), stage_s = smem_u32(stage_out);
  // stage s of this launch's ring: A hi, B hi, then (three products) A lo, B lo; every tile starts on
  // a 16 KiB boundary, as the 128-byte swizzle wants
  auto a_hi = [&](int s) { return ring + static_cast<uint32_t>(s) * st_bytes; };
  auto b_hi = [&](int s) { return a_hi(s) + A_TILE; };
  auto a_lo = [&](int s) { return a_hi(s) + A_TILE + B_TILE; };
  auto b_lo = [&](int s) { return a_hi(s) + 2 * A_TILE + B_TILE; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES_SINGLE; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 4);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: the ring runs on across work units ----
    int last_round[STAGES_SINGLE];
    for (int s = 0; s < STAGES_SINGLE; ++s) last_round[s] = -1;
    int s = 0, r = 0;  // ring stage and round of the next k block
    bool stop = false;
    for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
      int m0, n0, z, kb0, nkb;
      coords(u, &m0, &n0, &z);
      if (n0 >= ncols) continue;
      krange(z, &kb0, &nkb);
      for (int kb = 0; kb < nkb; ++kb) {
        if (r >= 1 && !mbar_wait(empty0 + 8 * s, (r - 1) & 1, lim)) {
          atomicCAS(g.err, 0, ERR_WAIT_MMA);
          atomicExch(fail, 1);
          stop = true;
          break;
        }
        if (*(volatile int*)fail) {
          stop = true;
          break;
        }
        const int kc = (kb0 + kb) * BK;
        mbar_expect_tx(full0 + 8 * s, st_bytes);
        if (!(g.withhold && blockIdx.x == 0 && r == 0 && s == 0)) {  // (self-check: the first copies withheld)
          tma_load_2d(a_hi(s), &tA_hi, full0 + 8 * s, kc, m0);
          tma_load_2d(b_hi(s), &tB_hi, full0 + 8 * s, kc, n0);
          if (three) {
            tma_load_2d(a_lo(s), &tA_lo, full0 + 8 * s, kc, m0);
            tma_load_2d(b_lo(s), &tB_lo, full0 + 8 * s, kc, n0);
          }
          last_round[s] = r;
        }
        if (++s == nst) s = 0, ++r;
      }
    }
    // on an error path, let the copies already issued land before the CTA releases its memory
    if (*(volatile int*)fail)
      for (int q = 0; q < nst; ++q)
        if (last_round[q] >= 0) (void)mbar_wait(full0 + 8 * q, last_round[q] & 1, lim);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: unit i accumulates into TMEM columns (i & 1) * BN ----
    // One loop per product count, descriptors advanced by tile offsets (as in the two-SM kernel).
    auto mma_role = [&](auto three_c) {
      constexpr bool THREE = decltype(three_c)::value;
      constexpr uint32_t id = idesc<KIND>(BM, BN);
      constexpr uint32_t ST16 = (THREE ? STAGE_BYTES : A_TILE + B_TILE) >> 4;
      constexpr int NST = THREE ? STAGES : STAGES_SINGLE;
      constexpr uint32_t O_BH = A_TILE >> 4, O_AL = (A_TILE + B_TILE) >> 4, O_BL = (2 * A_TILE + B_TILE) >> 4;
      const uint64_t d_ring = sw128_desc(ring);
      uint64_t sd = d_ring;  // stage s
      int s = 0, r = 0;      // ring stage and round of the next k block
      int i = 0;
      bool stop = false;
      for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
        int m0, n0, z, kb0, nkb;
        coords(u, &m0, &n0, &z);
        if (n0 >= ncols) continue;
        krange(z, &kb0, &nkb);
        const int b = i & 1, use = i >> 1;
        if (use >= 1 && !mbar_wait(acce0 + 8 * b, (use - 1) & 1, lim)) {  // the epilogue has drained buffer b
          atomicCAS(g.err, 0, ERR_WAIT_ACC);
          atomicExch(fail, 1);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + static_cast<uint32_t>(b * BN);
        int issued = 0;
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(full0 + 8 * s, r & 1, lim)) {
            atomicCAS(g.err, 0, ERR_WAIT_TMA);
            atomicExch(fail, 1);
            stop = true;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < BK_BYTES / 32; ++kk) {  // 32 bytes of k per MMA: +2 in the address field
            const uint64_t ah = sd + 2 * kk, bh = sd + O_BH + 2 * kk;
            umma<KIND>(d, ah, bh, id, issued);
            if constexpr (THREE) {
              umma<KIND>(d, ah, sd + O_BL + 2 * kk, id, 1);
              umma<KIND>(d, sd + O_AL + 2 * kk, bh, id, 1);
            }
            issued = 1;
          }
          umma_commit(empty0 + 8 * s);
          if (++s == NST) {
            s = 0, ++r;
            sd = d_ring;
          } else {
            sd += ST16;
          }
        }
        if (stop) break;
        umma_commit(accf0 + 8 * b);  // fires once the unit's MMAs have completed
        ++i;
      }
    };
    if (three) mma_role(std::true_type{});
    else mma_role(std::false_type{});
    umma_commit(drain);  // fires once every MMA issued above has completed: TMEM may be released
    (void)mbar_wait(drain, 0, lim);
  } else if (warp >= 4) {
    // ---- epilogue: TMEM -> registers -> problem-major FP32 rows, 64 columns at a time ----
    const int q = warp & 3, et = threadIdx.x - 128;
    int i = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
      int m0, n0, z;
      coords(u, &m0, &n0, &z);
      if (n0 >= ncols) continue;
      const int b = i & 1, use = i >> 1;
      const bool ok = mbar_wait(accf0 + 8 * b, use & 1, lim);
      if (!ok) atomicCAS(g.err, 0, ERR_WAIT_ACC);
      if (bar_or_epi(!ok || *(volatile int*)fail)) {  // the four warps leave together
        atomicExch(fail, 1);
        break;
      }
      tc_fence_after();
      const uint32_t tq = tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(b * BN);
      // once every TMEM read of buffer b is done, hand it back to the MMA warp
      epilogue_tile(g, g.out + z * g.split_stride, tq, stage_out, stage_s, m0, n0, ncols, q, lane, et,
                    [&] { if (lane == 0) mbar_arrive(acce0 + 8 * b); });
      ++i;
    }
    if (g.bulk && et < 64) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---- two-SM variant (cta_group::2) of the same GEMM ---------------------------------------------
// A cluster of two CTAs (an SM pair) computes a 256 x 128 output tile (hi/lo launches) or a 256 x 256
// tile (single-product launches). Each CTA stages its own 128 rows of A and half of the tile's B
// rows; the even CTA issues M = 256 MMAs that read both CTAs' shared memory and accumulate into both
// CTAs' TMEM (each CTA's 128 rows x all the tile's columns). Per k block a CTA so stages 48 KiB
// (hi/lo: A hi, 64 B rows hi, A lo, B lo) for 128 x 128 of tensor work, 4 stages in its 192 KiB ring,
// or 32 KiB (A hi, 128 B rows hi) for 128 x 256 of work, 6 stages: twice the work per staged byte of
// the one-SM kernel's single product, whose launches are bound by the latency of their ring.
//   both CTAs, warp 0 lane 0: TMA producer into its own ring; the copies complete on the even CTA's
//                             "full" barriers (which expect both CTAs' bytes)
//   even CTA, warp 1 lane 0 : MMA issuer; its commits reach the "empty" and "accumulator full"
//                             barriers of both CTAs
//   both CTAs, warps 4..7   : epilogue of the CTA's own TMEM rows; the release of a TMEM buffer is
//                             counted on the even CTA (4 warps x 2 CTAs)
// Every mbarrier wait is bounded as in the one-SM kernel; the two cluster barriers (after set-up,
// before TMEM is released) are reached by every thread of both CTAs on every path.
constexpr int P_BM = 2 * BM;                                   // output rows per pair tile
constexpr int P_BNH = BN / 2;                                  // B rows staged by each CTA (hi/lo)
constexpr int P_B_TILE = P_BNH * BK_BYTES;                     // 8 KiB
constexpr int P_STAGE = 2 * A_TILE + 2 * P_B_TILE;             // 48 KiB: A hi, B hi, A lo, B lo
constexpr int P_STAGES = STAGES * STAGE_BYTES / P_STAGE;       // 4
constexpr int P_BN_SINGLE = 2 * BN;                            // pair tile columns, single product
constexpr int P_STAGE_SINGLE = A_TILE + 2 * P_B_TILE;          // 32 KiB: A hi, 128 B rows hi
constexpr int P_STAGES_SINGLE = STAGES * STAGE_BYTES / P_STAGE_SINGLE;  // 6
constexpr int P_STAGES_MAX = P_STAGES > P_STAGES_SINGLE ? P_STAGES : P_STAGES_SINGLE;
constexpr int P_NBARS = 2 * P_STAGES_MAX + 5;
constexpr uint32_t P_TMEM_COLS = 2 * P_BN_SINGLE;              // two accumulators of up to 256 columns
constexpr int P_GROUP_M = 8;                                   // row tiles per raster group
constexpr int P_SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + EPI_BYTES + P_NBARS * 8 + 16;
static_assert(P_SMEM_BYTES <= 232448, "shared memory per CTA");
static_assert(P_STAGE * P_STAGES <= STAGES * STAGE_BYTES && P_STAGE_SINGLE * P_STAGES_SINGLE <= STAGES * STAGE_BYTES,
              "ring");

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// The shared::cluster address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on a barrier that arrivals from the other CTA of the cluster complete.
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, unsigned long long lim = WAIT_NS) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait_cluster(bar, parity))
    if (global_ns() - t0 > lim) return false;
  return true;
}
// Tile load into this CTA's shared memory whose completion is counted on `bar` (a shared::cluster
// address: here the even CTA's barrier).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}
template <int KIND>
__device__ __forceinline__ void umma_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t id,
                                          uint32_t accumulate) {
  if constexpr (KIND == KIND_BF16)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(id), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(id), "r"(accumulate)
        : "memory");
}
// Arrive on the barrier at the same offset in both CTAs once the pair MMAs issued so far complete.
__device__ __forceinline__ void umma_commit_pair_both(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(static_cast<uint16_t>(3))
      : "memory");
}
__device__ __forceinline__ void umma_commit_pair(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

template <int KIND>
__global__ void __launch_bounds__(THREADS, 1)
    gemm3_pair_kernel(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
                      const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo,
                      const __grid_constant__ CUtensorMap tB_hi2, GemmArgs g) {
  constexpr int BK = KindTraits<KIND>::BK;
  extern __shared__ uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool even = rank == 0;
  const int pair = static_cast<int>(blockIdx.x >> 1), npairs = static_cast<int>(gridDim.x >> 1);
  const int ncols = g.n_cols ? *g.n_cols : g.N;
  const bool three = !g.hilo || *g.hilo != 0;
  const int nst = three ? P_STAGES : P_STAGES_SINGLE;
  const int bnp = three ? BN : P_BN_SINGLE, bnh = bnp / 2;  // pair tile columns, B rows per CTA
  const unsigned long long lim = g.wait_ns ? g.wait_ns : WAIT_NS;
  const uint32_t st_bytes = three ? P_STAGE : P_STAGE_SINGLE;
  const int mt = (g.M + P_BM - 1) / P_BM, nt = (g.N + bnp - 1) / bnp;
  const int units = mt * nt;
  const int nkb = (g.Kd + BK - 1) / BK;
  // pair tile u: groups of P_GROUP_M row tiles, m fastest within a group, so that the pairs at work
  // at one time share a band of A rows (2048 rows = 32 MiB of hi/lo BF16 at n = 4096) that stays in
  // L2 while the B tiles stream, instead of all of A (which L2 does not hold across waves)
  auto coords = [&](int u, int* m0, int* n0) {
    const int per = P_GROUP_M * nt, grp = u / per, r = u - grp * per;
    const int first = grp * P_GROUP_M, gsz = min(mt - first, P_GROUP_M);
    *m0 = (first + r % gsz) * P_BM;
    *n0 = (r / gsz) * bnp;
  };

  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* const stage_out = reinterpret_cast<float*>(base + STAGES * STAGE_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES + EPI_BYTES);
  // full[P_STAGES_MAX], empty[P_STAGES_MAX], acc_full[2], acc_empty[2], drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + P_NBARS);
  int* fail = reinterpret_cast<int*>(tmem_slot + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + P_STAGES_MAX);
  const uint32_t accf0 = smem_u32(bars + 2 * P_STAGES_MAX), acce0 = smem_u32(bars + 2 * P_STAGES_MAX + 2);
  const uint32_t drain = smem_u32(bars + 2 * P_STAGES_MAX + 4);
  const uint32_t ring = smem_u32(base), stage_s = smem_u32(stage_out);
  // stage s: A hi (16 KiB), B hi (8 KiB; 16 KiB for the single product's 128 rows), then (hi/lo) A lo,
  // B lo; every tile on a 1 KiB (8-row atom) boundary, at the same offsets in both CTAs (the pair MMAs
  // address the other CTA's tiles by this CTA's offsets)
  auto a_hi = [&](int s) { return ring + static_cast<uint32_t>(s) * st_bytes; };
  auto b_hi = [&](int s) { return a_hi(s) + A_TILE; };
  auto a_lo = [&](int s) { return a_hi(s) + A_TILE + P_B_TILE; };
  auto b_lo = [&](int s) { return a_hi(s) + 2 * A_TILE + P_B_TILE; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES_MAX; ++s) {
      mbar_init(full0 + 8 * s, 1);   // the even CTA's producer; the bytes of both CTAs' copies
      mbar_init(empty0 + 8 * s, 1);  // the pair MMAs' commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 8);  // one arrival per epilogue warp of either CTA
    }
    mbar_init(drain, 1);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // the pair allocates together: the same columns in both CTAs' TMEM
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(P_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // both CTAs' barriers are initialised before either CTA signals the other's
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer (both CTAs): this CTA's A rows and B rows of each pair tile ----
    const uint32_t full_even = mapa_rank(full0, 0);
    int last_round[P_STAGES_MAX];
    for (int s = 0; s < P_STAGES_MAX; ++s) last_round[s] = -1;
    const CUtensorMap* mb_hi = three ? &tB_hi : &tB_hi2;  // boxes of 64 or 128 B rows
    int s = 0, r = 0;
    bool stop = false;
    for (int u = pair; u < units && !stop; u += npairs) {
      int m0, n0;
      coords(u, &m0, &n0);
      if (n0 >= ncols) continue;
      const int ma = m0 + static_cast<int>(rank) * BM, nb = n0 + static_cast<int>(rank) * bnh;
      for (int kb = 0; kb < nkb; ++kb) {
        if (r >= 1 && !mbar_wait(empty0 + 8 * s, (r - 1) & 1, lim)) {
          atomicCAS(g.err, 0, ERR_WAIT_MMA);
          atomicExch(fail, 1);
          stop = true;
          break;
        }
        if (*(volatile int*)fail) {
          stop = true;
          break;
        }
        const int kc = kb * BK;
        const uint32_t fb = full_even + 8 * s;
        if (even) mbar_expect_tx(full0 + 8 * s, 2 * st_bytes);
        if (!(g.withhold && blockIdx.x == 0 && r == 0 && s == 0)) {  // (self-check: the first copies withheld)
          tma_load_2d_pair(a_hi(s), &tA_hi, fb, kc, ma);
          tma_load_2d_pair(b_hi(s), mb_hi, fb, kc, nb);
          if (three) {
            tma_load_2d_pair(a_lo(s), &tA_lo, fb, kc, ma);
            tma_load_2d_pair(b_lo(s), &tB_lo, fb, kc, nb);
          }
          last_round[s] = r;
        }
        if (++s == nst) s = 0, ++r;
      }
    }
    if (*(volatile int*)fail) {
      if (even) {  // let the copies already issued land before the CTA releases its memory
        for (int q = 0; q < nst; ++q)
          if (last_round[q] >= 0) (void)mbar_wait(full0 + 8 * q, last_round[q] & 1, lim);
      } else {  // this CTA's copies complete on the even CTA's barriers: give them 100 us to land
        const unsigned long long t0 = global_ns();
        while (global_ns() - t0 < 100000ull) __nanosleep(1000);
      }
    }
  } else if (warp == 1 && lane == 0 && even) {
    // ---- MMA issuer (even CTA): pair tile i accumulates into TMEM columns (i & 1) * BN ----
    // One loop per product count (a compile-time constant in each), with the smem descriptors
    // advanced by adding tile offsets in 16-byte units (the start-address field holds address / 16
    // of shared memory below 256 KiB, so the offsets add without carry).
    auto mma_role = [&](auto three_c) {
      constexpr bool THREE = decltype(three_c)::value;
      constexpr int NPT = THREE ? BN : P_BN_SINGLE;  // pair tile columns
      constexpr uint32_t id = idesc<KIND>(P_BM, NPT);
      constexpr uint32_t ST16 = (THREE ? P_STAGE : P_STAGE_SINGLE) >> 4;
      constexpr int NST = THREE ? P_STAGES : P_STAGES_SINGLE;
      constexpr uint32_t O_BH = A_TILE >> 4, O_AL = (A_TILE + P_B_TILE) >> 4, O_BL = (2 * A_TILE + P_B_TILE) >> 4;
      const uint64_t d_ring = sw128_desc(ring);
      uint64_t sd = d_ring;  // stage s
      int s = 0, r = 0, i = 0;
      bool stop = false;
      for (int u = pair; u < units && !stop; u += npairs) {
        int m0, n0;
        coords(u, &m0, &n0);
        if (n0 >= ncols) continue;
        const int b = i & 1, use = i >> 1;
        if (use >= 1 && !mbar_wait_cluster(acce0 + 8 * b, (use - 1) & 1, lim)) {  // both epilogues drained buffer b
          atomicCAS(g.err, 0, ERR_WAIT_ACC);
          atomicExch(fail, 1);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + static_cast<uint32_t>(b * NPT);
        int issued = 0;
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(full0 + 8 * s, r & 1, lim)) {
            atomicCAS(g.err, 0, ERR_WAIT_TMA);
            atomicExch(fail, 1);
            stop = true;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < BK_BYTES / 32; ++kk) {  // 32 bytes of k per MMA: +2 in the address field
            const uint64_t ah = sd + 2 * kk, bh = sd + O_BH + 2 * kk;
            umma_pair<KIND>(d, ah, bh, id, issued);
            if constexpr (THREE) {
              umma_pair<KIND>(d, ah, sd + O_BL + 2 * kk, id, 1);
              umma_pair<KIND>(d, sd + O_AL + 2 * kk, bh, id, 1);
            }
            issued = 1;
          }
          umma_commit_pair_both(empty0 + 8 * s);
          if (++s == NST) {
            s = 0, ++r;
            sd = d_ring;
          } else {
            sd += ST16;
          }
        }
        if (stop) break;
        umma_commit_pair_both(accf0 + 8 * b);
        ++i;
      }
    };
    if (three) mma_role(std::true_type{});
    else mma_role(std::false_type{});
    umma_commit_pair(drain);  // every pair MMA issued above has completed: TMEM may be released
    (void)mbar_wait(drain, 0, lim);
  } else if (warp >= 4) {
    // ---- epilogue (both CTAs): this CTA's 128 rows of each pair tile, 64 columns at a time ----
    const uint32_t acce_even = mapa_rank(acce0, 0);
    const int q = warp & 3, et = threadIdx.x - 128;
    int i = 0;
    for (int u = pair; u < units; u += npairs) {
      int m0, n0;
      coords(u, &m0, &n0);
      if (n0 >= ncols) continue;
      const int b = i & 1, use = i >> 1;
      const bool ok = mbar_wait(accf0 + 8 * b, use & 1, lim);
      if (!ok) atomicCAS(g.err, 0, ERR_WAIT_ACC);
      if (bar_or_epi(!ok || *(volatile int*)fail)) {
        atomicExch(fail, 1);
        break;
      }
      tc_fence_after();
      const int ma = m0 + static_cast<int>(rank) * BM;  // this CTA's rows of the pair tile
      const uint32_t tq = tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(b * bnp);
      // once every TMEM read of buffer b is done, count it on the even CTA; a 256-column tile
      // leaves as two 128-column halves
      auto release = [&] { if (lane == 0) mbar_arrive_remote(acce_even + 8 * b); };
      if (three) {
        epilogue_tile(g, g.out, tq, stage_out, stage_s, ma, n0, ncols, q, lane, et, release);
      } else {
        epilogue_tile(g, g.out, tq, stage_out, stage_s, ma, n0, ncols, q, lane, et, [] {});
        epilogue_tile(g, g.out, tq + BN, stage_out, stage_s, ma, n0 + BN, ncols, q, lane, et, release);
      }
      ++i;
    }
    if (g.bulk && et < 64) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // neither CTA releases TMEM or leaves while the other may still signal it
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P_TMEM_COLS) : "memory");
  }
}

// ---- host side: tensor maps through the driver entry point (no -lcuda link needed) ----
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D tensor map over rows x cols (row pitch `ld` elements), box = box_rows x one 128-byte k block.
// Elements past `cols` or `rows` read as zero.
template <int KIND>
inline bool make_map(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  constexpr int esize = KIND == KIND_BF16 ? 2 : 4;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * esize};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(KindTraits<KIND>::BK), static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = KIND == KIND_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  return fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 152;
  }
  return sms;
}

// Launch the three-term GEMM: A* [M][lda] (M x Kd used), B* [N][ldb] (N x Kd used); the row
// pitches are multiples of 16 bytes and the bases 16-byte aligned (checked by the map encoder).
// Internal linkage on purpose: every translation unit that includes this header registers its
// own copy of gemm3_kernel, and the dynamic shared-memory attribute has to be set on the copy
// that the unit launches, so each unit keeps its own "attribute set" flag.
template <int KIND>
static inline cudaError_t launch_gemm3(const void* A_hi, const void* A_lo, int lda, const void* B_hi, const void* B_lo,
                                int ldb, int M, int N, int Kd, const GemmArgs& args, cudaStream_t stream) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm3_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int nkb = (Kd + KindTraits<KIND>::BK - 1) / KindTraits<KIND>::BK;
  if (args.splits < 1 || args.splits > nkb) return cudaErrorInvalidValue;
  GemmArgs a = args;
  // column segments out + o * ld_out + m0 of M - m0 (<= 128) floats: 16-byte aligned and sized
  a.bulk = !a.store_direct && (reinterpret_cast<uintptr_t>(a.out) % 16 == 0) && a.ld_out % 4 == 0 &&
           M % 4 == 0 && (a.splits == 1 || a.split_stride % 4 == 0);
  CUtensorMap ta_hi, ta_lo, tb_hi, tb_lo;
  if (!make_map<KIND>(&ta_hi, A_hi, M, Kd, lda, BM) || !make_map<KIND>(&ta_lo, A_lo, M, Kd, lda, BM) ||
      !make_map<KIND>(&tb_hi, B_hi, N, Kd, ldb, BN) || !make_map<KIND>(&tb_lo, B_lo, N, Kd, ldb, BN))
    return cudaErrorInvalidValue;
  const long long units = static_cast<long long>((M + BM - 1) / BM) * ((N + BN - 1) / BN) * args.splits;
  const int grid = static_cast<int>(units < num_sms() ? units : num_sms());  // persistent: one CTA per SM
  gemm3_kernel<KIND><<<grid, THREADS, SMEM_BYTES, stream>>>(ta_hi, ta_lo, tb_hi, tb_lo, a);
  return cudaGetLastError();
}

// Launch the two-SM variant (same operands and arguments as launch_gemm3; no reduction split):
// clusters of two CTAs, as many pairs as can be resident at once (one CTA per SM), each taking
// 256 x 128 output tiles in turn.
template <int KIND>
static inline cudaError_t launch_gemm3_pair(const void* A_hi, const void* A_lo, int lda, const void* B_hi,
                                            const void* B_lo, int ldb, int M, int N, int Kd, const GemmArgs& args,
                                            cudaStream_t stream) {
  static bool attr = false;
  static int max_pairs = 0;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(gemm3_pair_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (args.splits != 1) return cudaErrorInvalidValue;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(THREADS, 1, 1);
  cfg.dynamicSmemBytes = P_SMEM_BYTES;
  cfg.stream = stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (!max_pairs) {
    cfg.gridDim = dim3(2 * (num_sms() / 2), 1, 1);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, gemm3_pair_kernel<KIND>, &cfg) != cudaSuccess || n < 1) {
      (void)cudaGetLastError();
      n = num_sms() / 2;
    }
    max_pairs = n < num_sms() / 2 ? n : num_sms() / 2;
  }
  GemmArgs a = args;
  a.bulk = !a.store_direct && (reinterpret_cast<uintptr_t>(a.out) % 16 == 0) && a.ld_out % 4 == 0 && M % 4 == 0;
  CUtensorMap ta_hi, ta_lo, tb_hi, tb_lo, tb_hi2;
  if (!make_map<KIND>(&ta_hi, A_hi, M, Kd, lda, BM) || !make_map<KIND>(&ta_lo, A_lo, M, Kd, lda, BM) ||
      !make_map<KIND>(&tb_hi, B_hi, N, Kd, ldb, P_BNH) || !make_map<KIND>(&tb_lo, B_lo, N, Kd, ldb, P_BNH) ||
      !make_map<KIND>(&tb_hi2, B_hi, N, Kd, ldb, P_BN_SINGLE / 2))
    return cudaErrorInvalidValue;
  const long long units = static_cast<long long>((M + P_BM - 1) / P_BM) * ((N + BN - 1) / BN);
  const int pairs = static_cast<int>(units < max_pairs ? units : max_pairs);
  cfg.gridDim = dim3(2 * pairs, 1, 1);
  return cudaLaunchKernelEx(&cfg, gemm3_pair_kernel<KIND>, ta_hi, ta_lo, tb_hi, tb_lo, tb_hi2, a);
}

// Splits of a reduction of `nkb` k blocks over `tiles` output tiles that minimise
// (work units per SM, rounded up) x (k blocks per split), at most 16.
inline int choose_splits(int tiles, int nkb) {
  const int sms = num_sms();
  int best = 1;
  long long best_cost = -1;
  for (int s = 1; s <= 16 && s <= nkb; ++s) {
    const long long waves = (static_cast<long long>(tiles) * s + sms - 1) / sms;
    const long long cost = waves * ((nkb + s - 1) / s);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = s;
    }
  }
  return best;
}

}  // namespace tc
}  // namespace otlm
