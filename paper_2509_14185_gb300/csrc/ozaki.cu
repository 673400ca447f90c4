// Split-precision (Ozaki) GEMM on the tcgen05 tensor cores: C op= A B^T with
// FP64 operands split into BF16 slices.  Used for the three dense
// contractions of the Gauss-Newton step (Methods, "Second-order Optimizer"):
// the Gram product G = J~^T J~, the CCF Hilbert contraction J_U = K J_g, and
// the trailing updates of the blocked Cholesky factorisation.  GB300 runs
// BF16 on its tensor cores ~1600x faster than FP64, so the FP64 values are
// split and the slice products accumulated exactly (Ozaki, Ogita, Oishi &
// Rump, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer. Algorithms
// 2012):
//
//  1. scale: each output index j (a column of a K x n operand, or a row of an
//     n x K operand) gets e_j with max_k |X_kj| < 2^{e_j}; scaling is exact;
//  2. digits: v = round(X_kj 2^{8S - e_j}) as a 64-bit integer, written as S
//     balanced base-256 digits a_1..a_S (|a_1| <= 256, |a_t| <= 128); slice t
//     holds a_t 2^{-8t}, exactly representable in BF16 (8-bit significand);
//  3. products: slice pairs (s, t) with s + t <= S + 1, grouped by level
//     l = s + t.  Within a level every product is an integer times 2^{-8l};
//     over a 128-long K chunk the integer partial sums stay below 2^24, so the
//     FP32 accumulation in tensor memory is exact for levels 2, 3, 4; those
//     are flushed after each chunk into double-FP32 (hi, lo) registers.
//     Levels >= 5 share one accumulator over the whole K range.
//  4. C_ij op= 2^{e_i + e_j} (hi + lo), in FP64.
// Entrywise error, scaled units x = X 2^{-e} (|x| < 1), K the contraction length:
//   2^{-8S-1} (|x_i|_1 + |x_j|_1) + K 2^{-16S-2} + K S(S-1)/2 2^{-8S-2}
//   + [S >= 4] (K_pad/16) 2^{-48} K S       (the last term: FP32 tail accumulator).
//
// Kernel (one 128 x 128 output tile per CTA, 320 threads): warp 0 issues TMA
// loads of the 2 S slice tiles of each 32-wide K stage into a shared-memory
// ring (64-byte swizzle); warp 1 allocates the 512 tensor-memory columns and
// one lane issues tcgen05.mma (M = N = 128, K = 16, BF16 in, FP32 accumulate)
// into four 128-column accumulators (levels 2, 3, 4, tail); warps 2..9 read
// them with tcgen05.ld (warp w: lanes 32 (w % 4) .. + 31, columns
// 64 ((w - 2) / 4) .. + 63) and own the double-FP32 sums; at the end the
// operand ring is reused to park the tile for coalesced FP64 stores.  Every
// mbarrier wait is bounded in time; a timeout sets bit 1 of the status word
// and the CTA drains its copies and MMAs and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gn_internal.cuh"

namespace gn {
namespace {

constexpr int TM = 128;            // output tile rows
constexpr int TN = 128;            // output tile cols (the default tile; BN = 64 halves it)
constexpr int BKS = 32;            // K per stage (64-byte rows, SWIZZLE_64B)
constexpr int SPC = 4;             // stages per exact-accumulation chunk (K = 128)
constexpr int SLICE_BYTES = TM * BKS * 2;   // one 128-row slice tile: 8 KB
constexpr int NTHREADS = 320;      // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr unsigned long long kWaitNs = 4000000000ull;   // default bound on any wait: 4 s

// one pipeline stage: S slices of A (TM rows) and S of B (BN rows), BKS wide
__host__ __device__ constexpr int stage_bytes(int S, int BN) { return S * (TM + BN) * BKS * 2; }
__host__ __device__ constexpr int n_stages(int S, int BN) {
  return (stage_bytes(S, BN) * 4 <= 200 * 1024) ? 4 : (stage_bytes(S, BN) * 3 <= 200 * 1024) ? 3 : 2;
}
// The operand ring is reused at the end to park the (hi, lo) tile; the
// mbarriers live after whichever of the two is larger.
__host__ __device__ constexpr int park_bytes(int BN) { return TM * (BN + 1) * 8; }
__host__ __device__ constexpr int bar_offset(int S, int BN) {
  return n_stages(S, BN) * stage_bytes(S, BN) > park_bytes(BN) ? n_stages(S, BN) * stage_bytes(S, BN)
                                                                : park_bytes(BN);
}

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: returns false (and raises bit 1 of the status word) after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* flag, unsigned long long limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (!mbar_try(bar, parity)) {
    if (now_ns() - t0 > limit_ns) {
      atomicOr(flag, 2);
      return false;
    }
  }
  return true;
}
// AND of a predicate over the 256 epilogue threads (named barrier 1): every one of them takes
// the same branch afterwards, so all run the same sequence of named-barrier syncs
__device__ __forceinline__ bool epilogue_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.b32 p, %1, 0;\n bar.red.and.pred q, 1, 256, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// K-major operand tile, rows of 64 bytes with the 64-byte swizzle; 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, N = BN, M = 128.
template <int BN>
constexpr uint32_t idesc_for() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}
template <int BN>
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc_for<BN>()), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}
// (hi, lo) += v in double-FP32: TwoSum (Knuth) puts the exact rounding error of
// hi + v into lo; lo stays ~2^-24 |hi| per add, so no renormalisation is needed
// before the final (double) hi + (double) lo.  Intrinsics keep the order.
__device__ __forceinline__ void dd_add(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
  lo = __fadd_rn(lo, err);
  hi = s;
}
// 2^e as a double (exact); the bit construction covers the normal range.
__device__ __forceinline__ double pow2(int e) {
  return (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52) : ldexp(1.0, e);
}
__device__ __forceinline__ float pow2f(int e) {
  return (e >= -126 && e <= 127) ? __int_as_float((e + 127) << 23) : ldexpf(1.0f, e);
}
// x 2^k as a double by integer operations on the bits: exact for a normal x and a normal
// result, with no FP64 instruction (GB300's FP64 pipe retires about two per clock per SM, so
// a conversion and a scaling multiply per element made the store loop FP64-bound); zero,
// subnormal or non-finite x and results outside the normal range take the FP64 path.
__device__ __forceinline__ double f2d_scaled(float x, int k) {
  const unsigned b = __float_as_uint(x);
  const int ex = (int)((b >> 23) & 0xff);
  const int e = ex - 127 + k + 1023;
  if (ex == 0 || ex == 0xff || e <= 0 || e >= 2047) return (double)x * pow2(k);
  return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) | ((unsigned long long)e << 52) |
                                          ((unsigned long long)(b & 0x7fffffu) << 29)));
}
// (u.x, u.y) += (h, l), both double-FP32 (TwoSum, then Fast2Sum renormalisation)
__device__ __forceinline__ void dd2_add(float2& u, float h, float l) {
  const float s = __fadd_rn(u.x, h);
  const float bb = __fsub_rn(s, u.x);
  const float err = __fadd_rn(__fsub_rn(u.x, __fsub_rn(s, bb)), __fsub_rn(h, bb));
  const float t = __fadd_rn(__fadd_rn(u.y, l), err);
  const float hi = __fadd_rn(s, t);
  u.y = __fsub_rn(t, __fsub_rn(hi, s));
  u.x = hi;
}
// Level of a slice pair and its tensor-memory slot: levels 2, 3, 4 -> slots 0, 1, 2; >= 5 -> 3.
__device__ __forceinline__ int slot_of(int s, int t) {
  const int l = s + t + 2;  // s, t are 0-based
  return l <= 4 ? l - 2 : 3;
}

struct OzArgs {
  int64_t rowsA, rowsB;   // rows per slice of A and B in their 2D slice views (padded)
  int64_t Kpad;           // padded contraction length (multiple of 32)
  int64_t M, N;           // valid output rows / cols
  int nt;                 // column tiles (rectangular decode)
  const int* eA;          // exponents of A rows (padded)
  const int* eB;          // exponents of B rows (padded)
  int64_t estride;        // chunked exponents: stride between the chunks' exponent arrays
  int spc;                // stages per flush chunk (SPC, or the exponent chunk)
  double* C;
  int64_t ldc;
  int mode;               // 0: C = v, 1: C += rs_i v, 2: C -= v, 3: C2 += v in double-FP32 (FP32 pipe)
  const double* rowscale; // mode 1 (may be null: 1)
  int* flag;
  // split-K: CTA b works on tile b / ksplit, flush chunks [(b % ksplit) cps, + cps) of the
  // contraction, and writes its unscaled (hi, lo) tile to part (null: no split, epilogue in place)
  int ksplit;
  int cps;
  float2* part;
  // tile range (sym): the launch computes tiles [tile0, tile0 + grid / ksplit) of the mt-square
  // lower triangle, numbered row by row or (colmajor) column by column
  int64_t tile0;
  int64_t mt;
  int colmajor;
  unsigned long long wait_ns;   // bound on every mbarrier wait
  int starve;                   // testing: the producer issues no copy, so the waits run out
};

// Blocked order of a whole lower triangle (order 2): the tiles in square super-blocks of
// kRasterSB x kRasterSB tiles, super-blocks row by row (J <= I), tiles row by row inside each
// (the diagonal super-blocks lower-triangular).  The CTAs in flight (about one super-block) then
// share kRasterSB row bands of A and kRasterSB of B, read at nearly the same contraction
// position, so most band reads hit in L2 instead of DRAM (row order keeps ~2 row tiles but every
// column band in flight).  A bijection onto the triangle: only the order of the tiles changes.
constexpr int64_t kRasterSB = 12;
__device__ __forceinline__ void sym_tile_blocked(int64_t t, int64_t mt, int64_t& ti, int64_t& tj) {
  const int64_t sb = kRasterSB;
  int64_t I = 0, base = 0;
  for (;;) {   // super-row I: I off-diagonal blocks of hh x sb tiles, then the diagonal block
    const int64_t hh = (mt - I * sb < sb) ? mt - I * sb : sb;
    const int64_t cnt = I * hh * sb + hh * (hh + 1) / 2;
    if (t < base + cnt || (I + 1) * sb >= mt) {
      int64_t u = t - base;
      if (u < I * hh * sb) {
        const int64_t J = u / (hh * sb), v = u % (hh * sb);
        ti = I * sb + v / sb;
        tj = J * sb + v % sb;
      } else {
        u -= I * hh * sb;
        int64_t r = (int64_t)((sqrt(8.0 * (double)u + 1.0) - 1.0) * 0.5);
        while ((r + 1) * (r + 2) / 2 <= u) r++;
        while (r * (r + 1) / 2 > u) r--;
        ti = I * sb + r;
        tj = I * sb + (u - r * (r + 1) / 2);
      }
      return;
    }
    base += cnt;
    I++;
  }
}

// Lower-triangular tile t of an mt x mt tile grid.  Row order: row ti holds tiles
// ti (ti + 1) / 2 .. + ti.  Column order (colmajor = 1): column tj holds the next mt - tj tiles,
// so the first C(c) = c mt - c (c - 1) / 2 tiles are exactly the tile columns 0 .. c - 1.  It is
// row order read backwards on the triangle reflected about its anti-diagonal,
// (ti, tj) -> (mt - 1 - tj, mt - 1 - ti), which maps the lower triangle onto itself.  Blocked
// order (colmajor = 2): sym_tile_blocked.
__device__ __forceinline__ void sym_tile(int64_t t, int64_t mt, int colmajor, int64_t& ti, int64_t& tj) {
  if (colmajor == 2) {
    sym_tile_blocked(t, mt, ti, tj);
    return;
  }
  if (colmajor) t = mt * (mt + 1) / 2 - 1 - t;
  ti = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= t) ti++;
  while (ti * (ti + 1) / 2 > t) ti--;
  tj = t - ti * (ti + 1) / 2;
  if (colmajor) {
    const int64_t a = mt - 1 - tj, b = mt - 1 - ti;
    ti = a;
    tj = b;
  }
}

// Tile t of the lower part of G with 128-row, 64-column tiles (row order): row tile ti holds the
// 2 ti + 2 column tiles 0 .. 2 ti + 1 (those reaching the diagonal), so rows start at ti (ti + 1).
__device__ __forceinline__ void sym_tile_half(int64_t t, int64_t& ti, int64_t& tj) {
  ti = (int64_t)((sqrt(4.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) <= t) ti++;
  while (ti * (ti + 1) > t) ti--;
  tj = t - ti * (ti + 1);
}

// ---------------------------------------------------------------------------
// main kernel
// ---------------------------------------------------------------------------
template <int S, bool SYM, bool CH, int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    ozaki_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const OzArgs p) {
  static_assert(BN == TM || BN == TM / 2, "tiles are 128 x 128 or 128 x 64");
  constexpr int NST = n_stages(S, BN);
  constexpr int STAGE_BYTES = stage_bytes(S, BN);
  constexpr int SLICE_B = BN * BKS * 2;          // one B slice tile
  // Chunked exponents flush all four slots after every chunk, so the next chunk's MMAs would
  // wait for the flush; on 128 x 64 tiles two sets of slots fit the 512 tensor-memory columns
  // and alternate between chunks (the MMAs fill one while the epilogue flushes the other).
  constexpr int NACC = (CH && BN == TM / 2) ? 2 : 1;
  constexpr int TMEM_COLS = 4 * BN * NACC;       // four accumulator slots per set
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + bar_offset(S, BN));
  uint64_t* empty = full + NST;
  uint64_t* acc_full = empty + NST;              // [NACC]
  uint64_t* acc_empty = acc_full + NACC;         // [NACC]
  uint64_t* done = acc_empty + NACC;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int abort_cta;
  __shared__ int ecs[2][TM];       // exponents of this tile's rows (0) and columns (1)
  // chunked mode: 2^e of the rows and columns per chunk, double buffered (a stub otherwise)
  __shared__ float eccf[CH ? 2 : 1][2][CH ? TM : 1];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t ti, tj;
  const int64_t tb = p.tile0 + blockIdx.x / p.ksplit;   // output tile
  const int ksp = (int)(blockIdx.x % p.ksplit);
  if (SYM) {  // tiles reaching the lower triangle
    if (BN == TM) sym_tile(tb, p.mt, p.colmajor, ti, tj);
    else sym_tile_half(tb, ti, tj);
  } else {
    ti = tb / p.nt;
    tj = tb % p.nt;
  }
  const int spc = CH ? p.spc : SPC;   // a compile-time constant on the single-exponent path
  // this CTA's part of the contraction: flush chunks [c0, c0 + nchunk), stages [kt0, kt0 + nk)
  const int nk_all = (int)(p.Kpad / BKS);
  const int nchunk_all = (nk_all + spc - 1) / spc;
  const int c0 = ksp * p.cps;
  const int c1 = (c0 + p.cps < nchunk_all) ? c0 + p.cps : nchunk_all;
  const int kt0 = c0 * spc;
  const int nk = ((c1 * spc < nk_all) ? c1 * spc : nk_all) - kt0;
  const int nchunk = c1 - c0;
  int* flag = p.flag;

  if (threadIdx.x == 0) {
    abort_cta = 0;
    for (int i = 0; i < NST; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int b = 0; b < NACC; b++) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 8);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "n"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      const int rowA = (int)(ti * TM), rowB = (int)(tj * BN);
      int issued = 0;
      for (int kt = 0; kt < (p.starve ? 0 : nk); kt++) {
        const int st = kt % NST;
        if (kt >= NST) {
          if (!mbar_wait(&empty[st], ((kt / NST) - 1) & 1, flag, p.wait_ns)) {
            abort_cta = 1;
            break;
          }
        }
        if (*(volatile int*)&abort_cta) break;
        unsigned char* base = smem + st * STAGE_BYTES;
        mbar_expect_tx(&full[st], STAGE_BYTES);
#pragma unroll
        for (int s = 0; s < S; s++) {
          tma_load_2d(base + s * SLICE_BYTES, &tmA, (kt0 + kt) * BKS, (int)(s * p.rowsA) + rowA, &full[st]);
          tma_load_2d(base + S * SLICE_BYTES + s * SLICE_B, &tmB, (kt0 + kt) * BKS, (int)(s * p.rowsB) + rowB,
                      &full[st]);
        }
        issued = kt + 1;
      }
      // drain: every issued stage must land before the CTA may exit.  A stage that does not
      // land within the bound raises bit 2 as well (copies may still be in flight); the CTA
      // still releases its tensor memory below, since a CTA that exits holding it would block
      // every later allocation on this SM, and the host fails the call with GN_ERR_TIMEOUT.
      for (int kt = (issued > NST ? issued - NST : 0); kt < issued; kt++)
        if (!mbar_wait(&full[kt % NST], (kt / NST) & 1, flag, p.wait_ns)) atomicOr(flag, 4);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      bool mma_issued = false;
      for (int c = 0; c < nchunk && ok; c++) {
        const int q_end = (nk - c * spc) < spc ? (nk - c * spc) : spc;
        const int ab = (NACC == 2) ? (c & 1) : 0;            // this chunk's set of slots
        const uint32_t tacc = tmem + (uint32_t)(ab * 4 * BN);
        for (int q = 0; q < q_end && ok; q++) {
          const int kt = c * spc + q;
          const int st = kt % NST;
          if (!mbar_wait(&full[st], (kt / NST) & 1, flag, p.wait_ns)) { ok = false; break; }
          tc_fence_after();
          const uint32_t base = smem_u32(smem + st * STAGE_BYTES);
          // pass 0: tail levels (>= 5); pass 1: the exact head levels.  With one exponent
          // per row the tail accumulates over the whole K and the per-chunk flush does not
          // read it, so pass 0 overlaps the flush of the previous chunk and only pass 1
          // waits for it.  With chunked exponents every chunk flushes the tail too, so
          // both passes wait.
#pragma unroll
          for (int pass = 0; pass < 2; pass++) {
            // (two sets: the flush of chunk c - 2, which used the same set)
            if (q == 0 && c >= NACC && pass == (CH ? 0 : 1)) {
              const uint32_t par = (NACC == 2) ? (uint32_t)(((c >> 1) - 1) & 1) : (uint32_t)((c - 1) & 1);
              if (!mbar_wait(&acc_empty[ab], par, flag, p.wait_ns)) { ok = false; break; }
              tc_fence_after();
            }
#pragma unroll
            for (int s = 0; s < S; s++)
#pragma unroll
              for (int u = 0; u < S; u++) {
                if (s + u > S - 1) continue;  // keep levels s + t <= S + 1 (1-based)
                const int slot = slot_of(s, u);
                if ((slot == 3) != (pass == 0)) continue;
#pragma unroll
                for (int kk = 0; kk < BKS / 16; kk++) {
                  const uint64_t da = smem_desc(base + s * SLICE_BYTES + kk * 32);
                  const uint64_t db = smem_desc(base + S * SLICE_BYTES + u * SLICE_B + kk * 32);
                  // the first pair of a level (s = 0) resets the slot: per chunk for the
                  // exact head levels; for the tail once, or per chunk with chunked exponents
                  const bool first = (slot < 3) ? (q == 0 && kk == 0 && s == 0)
                                                : ((CH ? q : kt) == 0 && kk == 0 && s == 0 && u == 3);
                  mma_bf16<BN>(tacc + slot * BN, da, db, first ? 0u : 1u);
                  mma_issued = true;
                }
              }
          }
          if (!ok) break;
          mma_commit(&empty[st]);
        }
        if (ok) mma_commit(&acc_full[ab]);
      }
      if (!ok) abort_cta = 1;
      // every issued MMA must complete before tensor memory is released (nothing to wait for
      // when none was issued).  A timeout here raises bit 2 too; tensor memory is released all
      // the same (see the producer's drain) and the host fails the call with GN_ERR_TIMEOUT.
      if (mma_issued) {
        mma_commit(done);
        if (!mbar_wait(done, 0, flag, p.wait_ns)) atomicOr(flag, 4);
      }
    }
  } else {
    // ---------------- epilogue: 8 warps, BN / 2 columns each ----------------
    constexpr int EC = BN / 2;                  // columns per epilogue thread
    const int quad = warp & 3;
    const int qcol = (warp - 2) >> 2;          // column half 0..1
    const int row = quad * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(qcol * EC);
    // chunked exponents are applied at each chunk's flush, so the final scale is 2^0
    ecs[qcol][row] = (CH || (qcol == 1 && row >= BN)) ? 0 : ((qcol == 0) ? p.eA[ti * TM + row] : p.eB[tj * BN + row]);
    asm volatile("bar.sync 1, 256;" ::: "memory");   // the 8 epilogue warps only
    float hi[EC], lo[EC];
#pragma unroll
    for (int i = 0; i < EC; i++) { hi[i] = 0.f; lo[i] = 0.f; }
    constexpr int nhead = S < 3 ? S : 3;        // head levels present: 2..min(S+1, 4)
    bool ok = true;
    // Read-modify-write launches that are not the Gram (the factorisation's updates into U, the
    // Hilbert contraction into J): the final loop waits for the tile's old values; their lines
    // are fetched into L2 while the last two chunks' MMAs run, so that wait is an L2 latency
    // rather than a DRAM one (a tile row is BN x 8 bytes: 8 or 4 lines of 128 bytes).  Damped
    // solve 17.34 -> 16.98 ms, Jacobian phase 6.16 -> 6.10 ms; the symmetric single-exponent
    // build (the Gram, which stores without reading) is compiled without it.
    const int pfc = nchunk >= 2 ? nchunk - 2 : 0;
    for (int c = 0; c < nchunk; c++) {
      if constexpr (CH || !SYM) {
        if (c == pfc && p.mode != 0 && !p.part) {
          constexpr int LPR = BN * 8 / 128;         // lines per tile row
          const char* Cb = reinterpret_cast<const char*>(p.C);
          for (int l = (warp - 2) * 32 + lane; l < TM * LPR; l += 256) {
            const int r = l / LPR, seg = l % LPR;
            const int64_t gi = ti * TM + r, gj = tj * BN + seg * 16;
            if (gi < p.M && gj < p.N) prefetch_l2(Cb + (gi * p.ldc + gj) * 8);
          }
        }
      }
      if constexpr (CH) {
        // this chunk's exponents (double buffered: every thread has passed the previous
        // chunk's barrier, so nobody still reads the buffer of chunk c - 2)
        const int ev = (qcol == 0) ? p.eA[(c0 + c) * p.estride + ti * TM + row]
                                   : (row < BN ? p.eB[(c0 + c) * p.estride + tj * BN + row] : 0);
        eccf[c & 1][qcol][row] = pow2f(ev);
        asm volatile("bar.sync 1, 256;" ::: "memory");
      }
      // one decision for all 256 epilogue threads: a thread whose own bounded wait ran out
      // while another's succeeded must not leave the loop alone (the chunked path's in-loop
      // bar.sync and the one after the loop would then find too few partners)
      const int ab = (NACC == 2) ? (c & 1) : 0;
      const uint32_t par = (NACC == 2) ? (uint32_t)((c >> 1) & 1) : (uint32_t)(c & 1);
      const uint32_t lbase = lane_base + (uint32_t)(ab * 4 * BN);
      if (!epilogue_all(mbar_wait(&acc_full[ab], par, flag, p.wait_ns))) { ok = false; break; }
      tc_fence_after();
      if constexpr (CH) {
        // head levels and the tail, each scaled by this chunk's 2^e_row 2^e_col (two exact
        // power-of-two products; the scales come from shared memory, see below)
        const float rsc = eccf[c & 1][0][row];
#pragma unroll
        for (int slot = 0; slot < 4; slot++) {
          if (slot >= nhead && slot != 3) continue;
          if (slot == 3 && S < 4) continue;
#pragma unroll
          for (int part = 0; part < EC / 16; part++) {
            float v[16];
            tmem_ld16(lbase + (uint32_t)(slot * BN + part * 16), v);
#pragma unroll
            for (int i = 0; i < 16; i++)
              dd_add(hi[part * 16 + i], lo[part * 16 + i],
                     __fmul_rn(__fmul_rn(v[i], rsc), eccf[c & 1][1][qcol * EC + part * 16 + i]));
          }
        }
      } else {
#pragma unroll
        for (int slot = 0; slot < nhead; slot++) {
#pragma unroll
          for (int part = 0; part < EC / 16; part++) {
            float v[16];
            tmem_ld16(lbase + (uint32_t)(slot * BN + part * 16), v);
#pragma unroll
            for (int i = 0; i < 16; i++) dd_add(hi[part * 16 + i], lo[part * 16 + i], v[i]);
          }
        }
        if (S >= 4 && c == nchunk - 1) {
#pragma unroll
          for (int part = 0; part < EC / 16; part++) {
            float v[16];
            tmem_ld16(lbase + (uint32_t)(3 * BN + part * 16), v);
#pragma unroll
            for (int i = 0; i < 16; i++) dd_add(hi[part * 16 + i], lo[part * 16 + i], v[i]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[ab]);
    }
    // All loads have landed and all MMAs have completed (the last acc_full),
    // so the operand ring is free: park (hi, lo) there, then convert and store
    // the tile with coalesced writes.
    float2* park = reinterpret_cast<float2*>(smem);
    if (ok) {
#pragma unroll
      for (int i = 0; i < EC; i++) park[row * (BN + 1) + qcol * EC + i] = make_float2(hi[i], lo[i]);
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (ok && p.part) {
      // split-K partial: the unscaled (hi, lo) tile, coalesced; oz_splitk_reduce finishes it
      const int et = (warp - 2) * 32 + lane;
      float2* dst = p.part + (size_t)blockIdx.x * (TM * BN);
      for (int idx = et; idx < TM * BN; idx += 256) dst[idx] = park[(idx / BN) * (BN + 1) + (idx % BN)];
    } else if (ok) {
      // 64 elements per thread, in batches of 8 whose global loads are issued
      // together (a load-modify-store loop would expose one memory latency per element)
      const int et = (warp - 2) * 32 + lane;
      constexpr int B8 = 8;
      for (int base_i = 0; base_i < TM * BN / 256; base_i += B8) {
        int64_t off[B8];
        bool in[B8];
        float2 hl[B8];
        double cv[B8];
        float2 uv[B8];
        double rs[B8];
#pragma unroll
        for (int q = 0; q < B8; q++) {
          const int idx = et + (base_i + q) * 256;
          const int r = idx / BN, cc = idx % BN;
          const int64_t gi = ti * TM + r, gj = tj * BN + cc;
          in[q] = (gi < p.M && gj < p.N);
          off[q] = gi * p.ldc + gj;
          hl[q] = park[r * (BN + 1) + cc];
          if (p.mode == 3) hl[q] = make_float2(hl[q].x * pow2f(ecs[0][r] + ecs[1][cc]),
                                              hl[q].y * pow2f(ecs[0][r] + ecs[1][cc]));
          else {
            const int e = ecs[0][r] + ecs[1][cc];
            if constexpr (CH) {   // not reached: chunked launches accumulate into U (mode 3)
              cv[q] = ((double)hl[q].x + (double)hl[q].y) * pow2(e);
            } else {
              // (hi + lo) 2^e with one FP64 addition: the two scalings are exact bit operations
              // and rounding the sum commutes with them, so this equals (hi + lo rounded) 2^e
              cv[q] = f2d_scaled(hl[q].x, e) + f2d_scaled(hl[q].y, e);
            }
          }
          rs[q] = (p.mode == 1 && p.rowscale && in[q]) ? p.rowscale[gi] : 1.0;
        }
        if (p.mode == 3) {
          // accumulate without any FP64 arithmetic (GB300's FP64 rate is ~1/60 of FP32)
          float2* U = reinterpret_cast<float2*>(p.C);
#pragma unroll
          for (int q = 0; q < B8; q++) uv[q] = in[q] ? U[off[q]] : make_float2(0.f, 0.f);
#pragma unroll
          for (int q = 0; q < B8; q++)
            if (in[q]) {
              dd2_add(uv[q], hl[q].x, hl[q].y);
              U[off[q]] = uv[q];
            }
        } else if (p.mode == 0) {
#pragma unroll
          for (int q = 0; q < B8; q++)
            if (in[q]) p.C[off[q]] = cv[q];
        } else {
          double old[B8];
#pragma unroll
          for (int q = 0; q < B8; q++) old[q] = in[q] ? p.C[off[q]] : 0.0;
#pragma unroll
          for (int q = 0; q < B8; q++)
            if (in[q]) p.C[off[q]] = (p.mode == 1) ? fma(rs[q], cv[q], old[q]) : old[q] - cv[q];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS));
  }
}

// Split-K epilogue: C_ij op= 2^(e_i + e_j) sum_ks (hi + lo)_ks, the partial tiles summed in
// split order (deterministic), then the same store / add / subtract as the fused epilogue.
template <bool SYM, int BN>
__global__ void __launch_bounds__(256) oz_splitk_reduce(const float2* __restrict__ part, int ksplit, OzArgs p) {
  const int64_t tb = p.tile0 + blockIdx.x;
  int64_t ti, tj;
  if (SYM) {
    if (BN == TM) sym_tile(tb, p.mt, p.colmajor, ti, tj);
    else sym_tile_half(tb, ti, tj);
  } else {
    ti = tb / p.nt;
    tj = tb % p.nt;
  }
  const float2* src = part + (size_t)blockIdx.x * ksplit * (TM * BN);
  for (int idx = threadIdx.x; idx < TM * BN; idx += 256) {
    const int r = idx / BN, cc = idx % BN;
    const int64_t gi = ti * TM + r, gj = tj * BN + cc;
    if (gi >= p.M || gj >= p.N) continue;
    double v = 0.0;
    for (int k = 0; k < ksplit; k++) {
      const float2 hl = src[(size_t)k * (TM * BN) + idx];
      v += (double)hl.x + (double)hl.y;
    }
    const double cv = v * pow2(p.eA[gi] + p.eB[gj]);
    const int64_t off = gi * p.ldc + gj;
    if (p.mode == 0) p.C[off] = cv;
    else if (p.mode == 1) p.C[off] = fma(p.rowscale ? p.rowscale[gi] : 1.0, cv, p.C[off]);
    else p.C[off] = p.C[off] - cv;
  }
}

// ---------------------------------------------------------------------------
// operand preparation: exponents and slices (K-major, [S][npad][kpad] BF16)
// ---------------------------------------------------------------------------
// columns of a K x n row-major matrix (J layout): partial column maxima over 64 row chunks
constexpr int CM_CHUNKS = 64;
__global__ void colmax_partial(const double* __restrict__ X, int64_t ld, int64_t nrows, int64_t ncols,
                               double* part) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  const int c = blockIdx.y;
  const int64_t per = (nrows + CM_CHUNKS - 1) / CM_CHUNKS;
  const int64_t r0 = c * per, r1 = (r0 + per < nrows) ? r0 + per : nrows;
  // max |x| as the largest bit pattern of |x| (the order of non-negative doubles), NaNs skipped
  // as fmax skips them: integer operations, where fmax/fabs would run on the FP64 pipe
  unsigned long long m = 0;
  for (int64_t r = r0; r < r1; r++) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(X[r * ld + j]) & 0x7FFFFFFFFFFFFFFFull;
    if (a <= 0x7FF0000000000000ull && a > m) m = a;
  }
  part[(int64_t)c * ncols + j] = __longlong_as_double((long long)m);
}
__global__ void colexp_kernel(const double* __restrict__ part, int64_t ncols, int64_t npad, int* e) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= npad) return;
  int ex = 0;
  if (j < ncols) {
    double m = 0.0;
    for (int c = 0; c < CM_CHUNKS; c++) m = fmax(m, part[(int64_t)c * ncols + j]);
    if (m > 0.0 && isfinite(m)) frexp(m, &ex);  // m = f 2^ex, f in [0.5, 1): 2^ex > m
  }
  e[j] = ex;
}
// 64 rows x 32 columns per block, transposed through shared memory
template <int S>
__global__ void __launch_bounds__(256) split_cols_kernel(const double* __restrict__ X, int64_t ld, int64_t nrows,
                                                         int64_t ncols, const int* __restrict__ e, int64_t npad,
                                                         int64_t kpad, __nv_bfloat16* out) {
  __shared__ __align__(16) __nv_bfloat16 sl[S][32][64 + 8];
  const int t = threadIdx.x;
  const int64_t k0 = (int64_t)blockIdx.x * 64, j0 = (int64_t)blockIdx.y * 32;
  const int jj = t & 31;
  const int64_t j = j0 + jj;
  const int ex = (j < npad) ? e[j] : 0;
#pragma unroll
  for (int r = 0; r < 8; r++) {
    const int kk = (t >> 5) + 8 * r;
    const int64_t k = k0 + kk;
    const double x = (k < nrows && j < ncols) ? X[k * ld + j] : 0.0;
    oz_digits<S>(x, ex, &sl[0][jj][kk], 32 * (64 + 8));
  }
  __syncthreads();
  for (int idx = t; idx < S * 32 * 8; idx += 256) {
    const int q = idx / (32 * 8), rem = idx % (32 * 8);
    const int c = rem / 8, seg = rem % 8;
    const int64_t col = j0 + c;
    if (col >= npad || k0 + seg * 8 >= kpad) continue;
    const uint4 val = *reinterpret_cast<const uint4*>(&sl[q][c][seg * 8]);
    *reinterpret_cast<uint4*>(out + ((int64_t)q * npad + col) * kpad + k0 + seg * 8) = val;
  }
}
// rows of an n x K row-major matrix: one warp per row for the exponent
__global__ void rowexp_kernel(const double* __restrict__ X, int64_t ld, int64_t nrows, int64_t k, int64_t npad,
                              int* e) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= npad) return;
  double m = 0.0;
  if (row < nrows)
    for (int64_t c = lane; c < k; c += 32) m = fmax(m, fabs(X[row * ld + c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if (lane == 0) {
    int ex = 0;
    if (m > 0.0 && isfinite(m)) frexp(m, &ex);
    e[row] = ex;
  }
}
template <int S>
__global__ void split_rows_kernel(const double* __restrict__ X, int64_t ld, int64_t nrows, int64_t k,
                                  const int* __restrict__ e, int64_t npad, int64_t kpad, __nv_bfloat16* out) {
  const int64_t total = npad * kpad;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / kpad, c = idx - row * kpad;
    const double x = (row < nrows && c < k) ? X[row * ld + c] : 0.0;
    oz_digits<S>(x, e[row], out + row * kpad + c, npad * kpad);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  // looked up once; a function-local static is initialised thread-safely (batched
  // fits step their handles from several host threads)
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &ptr, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(ptr);
    return nullptr;
  }();
  return fn;
}

int64_t rup(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

int encode(const OzOperand& op, int S, CUtensorMap* map, int box_rows = TM) {
  EncodeTiledFn enc = get_encode();
  if (!enc) {
    set_detail(__FILE__, __LINE__, "cuTensorMapEncodeTiled entry point not found");
    return GN_ERR_UNSUPPORTED;
  }
  memset(map, 0, sizeof(*map));
  cuuint64_t dims[2] = {(cuuint64_t)op.kpad, (cuuint64_t)(op.map_rows > 0 ? op.map_rows : S * op.npad)};
  cuuint64_t strides[1] = {(cuuint64_t)(op.kpad * 2)};
  cuuint32_t box[2] = {BKS, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, op.slices, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    char msg[64];
    snprintf(msg, sizeof(msg), "cuTensorMapEncodeTiled returned %d", (int)cr);
    set_detail(__FILE__, __LINE__, msg);
    return GN_ERR_CUDA;
  }
  return GN_OK;
}

template <int S>
int prep_cols(const double* X, int64_t ld, int64_t k, int64_t n, const OzOperand& op, double* part,
              cudaStream_t st) {
  dim3 g((unsigned)((n + 127) / 128), CM_CHUNKS);
  colmax_partial<<<g, 128, 0, st>>>(X, ld, k, n, part);
  count_launch();
  colexp_kernel<<<(unsigned)((op.npad + 255) / 256), 256, 0, st>>>(part, n, op.npad, op.e);
  count_launch();
  dim3 gs((unsigned)((op.kpad + 63) / 64), (unsigned)(op.npad / 32));   // kpad is a multiple of 32
  split_cols_kernel<S><<<gs, 256, 0, st>>>(X, ld, k, n, op.e, op.npad, op.kpad,
                                          static_cast<__nv_bfloat16*>(op.slices));
  count_launch();
  return GN_NOTE(cudaGetLastError()) == cudaSuccess ? GN_OK : GN_ERR_CUDA;
}

template <int S>
int prep_rows(const double* X, int64_t ld, int64_t n, int64_t k, const OzOperand& op, cudaStream_t st) {
  rowexp_kernel<<<(unsigned)((op.npad * 32 + 255) / 256), 256, 0, st>>>(X, ld, n, k, op.npad, op.e);
  count_launch();
  int64_t blocks = (op.npad * op.kpad + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  split_rows_kernel<S><<<(unsigned)blocks, 256, 0, st>>>(X, ld, n, k, op.e, op.npad, op.kpad,
                                                         static_cast<__nv_bfloat16*>(op.slices));
  count_launch();
  return GN_NOTE(cudaGetLastError()) == cudaSuccess ? GN_OK : GN_ERR_CUDA;
}

}  // namespace

// Testing hooks of the bounded waits (gn_test_bounded_waits): the bound on every mbarrier wait
// of the split GEMM, and whether its producer issues no copies.
std::atomic<unsigned long long> g_oz_wait_ns{kWaitNs};
std::atomic<int> g_oz_starve{0};

namespace {

template <int S, bool SYM, int BN>
int launch_oz(const OzOperand& A, const OzOperand& B, int64_t M, int64_t N, double* C, int64_t ldc, int mode,
              const double* rowscale, int* flag, cudaStream_t st, int ksplit, void* part, const OzRange& range) {
  CUtensorMap ma, mb;
  int rc = encode(A, S, &ma, TM);
  if (rc) return rc;
  rc = encode(B, S, &mb, BN);
  if (rc) return rc;
  const size_t smem = (size_t)bar_offset(S, BN) + 1024 + 256;
  const bool ch = A.echunk > 0;
  if (GN_NOTE(cudaFuncSetAttribute(ch ? ozaki_kernel<S, SYM, true, BN> : ozaki_kernel<S, SYM, false, BN>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return GN_ERR_CUDA;
  OzArgs a;
  a.rowsA = A.npad;
  a.rowsB = B.npad;
  a.Kpad = A.kuse > 0 ? A.kuse : A.kpad;
  a.M = M;
  a.N = N;
  const int64_t mt = (M + TM - 1) / TM, nt = (N + BN - 1) / BN;
  a.nt = (int)nt;
  a.eA = A.e;
  a.eB = B.e;
  a.spc = A.echunk > 0 ? A.echunk / BKS : SPC;
  a.estride = A.estride;
  a.C = C;
  a.ldc = ldc;
  a.mode = mode;
  a.rowscale = rowscale;
  a.flag = flag;
  a.wait_ns = g_oz_wait_ns.load(std::memory_order_relaxed);
  a.starve = g_oz_starve.load(std::memory_order_relaxed);
  // sym: the tiles reaching the lower triangle (square tiles: mt (mt + 1) / 2; 64-column tiles:
  // 2 ti + 2 in row tile ti, mt (mt + 1) in all)
  const int64_t all_tiles = SYM ? (BN == TM ? mt * (mt + 1) / 2 : mt * (mt + 1)) : mt * nt;
  a.tile0 = 0;
  a.mt = mt;
  a.colmajor = (SYM && BN == TM) ? 2 : 0;   // a whole square-tile triangle: the blocked order
  int64_t tiles = all_tiles;
  if (range.ntiles >= 0) {   // a range of the triangle's tiles (sym only; column order: square tiles)
    if (!SYM || range.tile0 < 0 || range.tile0 + range.ntiles > all_tiles || (range.colmajor && BN != TM))
      return GN_ERR_INVALID;
    a.tile0 = range.tile0;
    a.colmajor = range.colmajor;
    tiles = range.ntiles;
  }
  if (tiles <= 0) return GN_OK;
  const int nchunk_all = (int)((a.Kpad / BKS + a.spc - 1) / a.spc);
  if (ksplit < 1 || ch || mode == 3 || !part) ksplit = 1;   // split-K: single-exponent modes 0-2 only
  a.cps = (nchunk_all + ksplit - 1) / ksplit;
  if (a.cps < 1) a.cps = 1;
  ksplit = (nchunk_all + a.cps - 1) / a.cps;   // no empty splits
  if (ksplit < 1) ksplit = 1;
  a.ksplit = ksplit;
  a.part = ksplit > 1 ? static_cast<float2*>(part) : nullptr;
  const unsigned grid = (unsigned)(tiles * ksplit);
  if (ch)
    ozaki_kernel<S, SYM, true, BN><<<grid, NTHREADS, smem, st>>>(ma, mb, a);
  else
    ozaki_kernel<S, SYM, false, BN><<<grid, NTHREADS, smem, st>>>(ma, mb, a);
  count_launch();
  if (ksplit > 1) {
    oz_splitk_reduce<SYM, BN><<<(unsigned)tiles, 256, 0, st>>>(a.part, ksplit, a);
    count_launch();
  }
  return GN_NOTE(cudaGetLastError()) == cudaSuccess ? GN_OK : GN_ERR_CUDA;
}

}  // namespace

size_t oz_operand_bytes(int S, int64_t n, int64_t k) {
  const int64_t npad = rup(n > 0 ? n : 1, TM), kpad = rup(k > 0 ? k : 1, BKS);
  return rup((size_t)S * npad * kpad * 2, 256) + rup((size_t)npad * sizeof(int), 256);
}

OzOperand oz_operand_at(void* base, int S, int64_t n, int64_t k) {
  OzOperand op;
  op.npad = rup(n > 0 ? n : 1, TM);
  op.kpad = rup(k > 0 ? k : 1, BKS);
  op.slices = static_cast<__nv_bfloat16*>(base);
  op.e = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + rup((size_t)S * op.npad * op.kpad * 2, 256));
  return op;
}

int oz_prepare_cols(int S, const double* X, int64_t ld, int64_t k, int64_t n, const OzOperand& op, double* part,
                    cudaStream_t st) {
  switch (S) {
    case 1: return prep_cols<1>(X, ld, k, n, op, part, st);
    case 2: return prep_cols<2>(X, ld, k, n, op, part, st);
    case 3: return prep_cols<3>(X, ld, k, n, op, part, st);
    case 4: return prep_cols<4>(X, ld, k, n, op, part, st);
    case 5: return prep_cols<5>(X, ld, k, n, op, part, st);
    case 6: return prep_cols<6>(X, ld, k, n, op, part, st);
    default: return GN_ERR_UNSUPPORTED;
  }
}

int oz_prepare_rows(int S, const double* X, int64_t ld, int64_t n, int64_t k, const OzOperand& op,
                    cudaStream_t st) {
  switch (S) {
    case 1: return prep_rows<1>(X, ld, n, k, op, st);
    case 2: return prep_rows<2>(X, ld, n, k, op, st);
    case 3: return prep_rows<3>(X, ld, n, k, op, st);
    case 4: return prep_rows<4>(X, ld, n, k, op, st);
    case 5: return prep_rows<5>(X, ld, n, k, op, st);
    case 6: return prep_rows<6>(X, ld, n, k, op, st);
    default: return GN_ERR_UNSUPPORTED;
  }
}

OzOperand oz_operand_rows(const OzOperand& op, int S, int64_t row_off) {
  OzOperand v = op;
  v.slices = static_cast<__nv_bfloat16*>(op.slices) + row_off * op.kpad;
  v.e = op.e + row_off;
  v.map_rows = (op.map_rows > 0 ? op.map_rows : S * op.npad) - row_off;
  return v;
}

int oz_gemm(int S, bool sym, const OzOperand& A, const OzOperand& B, int64_t M, int64_t N, double* C, int64_t ldc,
            int mode, const double* rowscale, int* flag, cudaStream_t st, int ksplit, void* part,
            const OzRange& range, int tile_n) {
  if (tile_n != TM && tile_n != TM / 2) return GN_ERR_INVALID;
  if (A.kpad != B.kpad || A.kuse != B.kuse || A.kuse % BKS != 0 || A.kuse > A.kpad) return GN_ERR_INVALID;
  if (A.echunk != B.echunk || A.estride != B.estride || A.echunk % BKS != 0 || A.echunk > SPC * BKS ||
      (A.echunk > 0 && A.estride <= 0))
    return GN_ERR_INVALID;
#define GN_OZ_CASE(s)                                                                                     \
  case s:                                                                                                 \
    if (tile_n == TM)                                                                                     \
      return sym ? launch_oz<s, true, TM>(A, B, M, N, C, ldc, mode, rowscale, flag, st, ksplit, part, range) \
                 : launch_oz<s, false, TM>(A, B, M, N, C, ldc, mode, rowscale, flag, st, ksplit, part, range); \
    return sym ? launch_oz<s, true, TM / 2>(A, B, M, N, C, ldc, mode, rowscale, flag, st, ksplit, part, range)  \
               : launch_oz<s, false, TM / 2>(A, B, M, N, C, ldc, mode, rowscale, flag, st, ksplit, part, range);
  switch (S) {
    GN_OZ_CASE(1)
    GN_OZ_CASE(2)
    GN_OZ_CASE(3)
    GN_OZ_CASE(4)
    GN_OZ_CASE(5)
    GN_OZ_CASE(6)
    default: return GN_ERR_UNSUPPORTED;
  }
#undef GN_OZ_CASE
}

int ensure_split_ws(gn_handle* h, size_t need) {
  if (h->split_ws_bytes >= need) return GN_OK;
  if (h->capturing) {   // prepare_for_capture sized it; growing now would allocate inside a capture
    set_detail(__FILE__, __LINE__, "split workspace would grow during a graph capture");
    return GN_ERR_UNSUPPORTED;
  }
  if (h->split_ws) cudaFree(h->split_ws);   // synchronises: no kernel still reads it
  h->split_ws = nullptr;
  h->split_ws_bytes = 0;
  if (GN_NOTE(cudaMalloc(&h->split_ws, need)) != cudaSuccess) return GN_ERR_OOM;
  h->split_ws_bytes = need;
  return GN_OK;
}

// ---------------------------------------------------------------------------
// Gram autotuner: tile shape and split-K.  A Gram of few tiles (small P') leaves most of the 152
// SMs idle; 128 x 64 tiles (twice as many CTAs, each with half the B operand and half the
// tensor memory) and cutting the contraction into ksplit parts both multiply the CTAs.  The
// best choice depends on the tile count, the contraction length and S, so it is measured: on
// the first split Gram of a shape (S, tile rows, flush chunks) every candidate (tile width,
// ksplit) is launched and timed with CUDA events, and the fastest is kept in a process-wide
// table (so every handle of that shape in the process takes the same, deterministic path).
// gn_set_gram_split and gn_set_gram_tile force one.
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t kSplitMaxCtas = 4 * 152;   // candidates keep tiles * ksplit within 4 waves
struct GramChoice {
  int ks = 1, tn = TN;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int64_t, int64_t>, GramChoice> g_tune;

int64_t gram_chunks(int64_t nrows) { return (rup(nrows > 0 ? nrows : 1, BKS) / BKS + SPC - 1) / SPC; }
int64_t gram_tiles(int64_t Pp, int tn = TN) {
  const int64_t mt = (Pp + TM - 1) / TM;
  return tn == TM ? mt * (mt + 1) / 2 : mt * (mt + 1);
}
std::vector<GramChoice> gram_candidates(gn_handle* h, int64_t nrows) {
  std::vector<GramChoice> c;
  const int64_t nch = gram_chunks(nrows);
  for (int tn : {TN, TN / 2}) {
    if (h->gram_tile > 0 && tn != h->gram_tile) continue;
    const int64_t tiles = gram_tiles(h->Pp, tn);
    if (h->gram_ksplit > 0) {
      c.push_back({h->gram_ksplit, tn});
      continue;
    }
    c.push_back({1, tn});
    int last = 1;
    for (int ks : {2, 3, 4, 6, 8}) {
      const int64_t cps = (nch + ks - 1) / ks;
      const int eff = (int)((nch + cps - 1) / cps);   // splits actually made
      if (tiles * eff > kSplitMaxCtas || cps < 2 || eff <= last) continue;
      c.push_back({eff, tn});
      last = eff;
    }
  }
  return c;
}
int gram_max_split(gn_handle* h, int64_t nrows) {
  int m = 1;
  for (const GramChoice& k : gram_candidates(h, nrows)) m = k.ks > m ? k.ks : m;
  return m;
}
// split-K partial tiles: the same bytes for either tile width (twice the tiles, half the size)
size_t gram_part_bytes(int64_t Pp, int ksplit) {
  return ksplit > 1 ? (size_t)gram_tiles(Pp) * ksplit * TM * TN * sizeof(float2) : 0;
}
bool lookup(int S, int64_t Pp, int64_t nrows, GramChoice* ch) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(S, (Pp + TM - 1) / TM, gram_chunks(nrows)));
  if (it == g_tune.end()) return false;
  *ch = it->second;
  return true;
}
// The choice a split Gram of this handle over nrows rows takes: forced, or tuned (false when the
// shape has not been tuned yet and nothing is forced).
bool gram_choice(gn_handle* h, int64_t nrows, GramChoice* ch) {
  GramChoice t;
  const bool tuned = lookup(h->n_slices, h->Pp, nrows, &t);
  if (h->gram_ksplit > 0 && h->gram_tile > 0) {
    *ch = {h->gram_ksplit, h->gram_tile};
    return true;
  }
  if (!tuned) return false;
  *ch = t;
  if (h->gram_ksplit > 0) ch->ks = h->gram_ksplit;
  if (h->gram_tile > 0) ch->tn = h->gram_tile;
  return true;
}
// Time every candidate on the prepared operand (mode 0 into C, which the caller overwrites
// afterwards) and record the fastest; the default (128-column tiles, no split) unless another
// wins by 3 %.  Synchronises the stream.
int tune(gn_handle* h, int S, const OzOperand& op, int64_t nrows, double* C, void* part, GramChoice* best_out) {
  const std::vector<GramChoice> cand = gram_candidates(h, nrows);
  GramChoice best = cand[0];
  if (cand.size() > 1) {
    cudaEvent_t e0, e1;
    if (GN_NOTE(cudaEventCreate(&e0)) != cudaSuccess) return GN_ERR_CUDA;
    if (GN_NOTE(cudaEventCreate(&e1)) != cudaSuccess) {
      cudaEventDestroy(e0);
      return GN_ERR_CUDA;
    }
    float best_ms = 0.f;
    int rc = GN_OK;
    bool first = true;
    for (const GramChoice& c : cand) {
      rc = oz_gemm(S, true, op, op, h->Pp, h->Pp, C, h->Pp, 0, nullptr, h->flag + 2, h->st, c.ks, part, OzRange(),
                   c.tn);   // warm
      if (rc) break;
      cudaEventRecord(e0, h->st);
      for (int r = 0; r < 3 && !rc; r++)
        rc = oz_gemm(S, true, op, op, h->Pp, h->Pp, C, h->Pp, 0, nullptr, h->flag + 2, h->st, c.ks, part,
                     OzRange(), c.tn);
      cudaEventRecord(e1, h->st);
      if (rc || GN_NOTE(cudaEventSynchronize(e1)) != cudaSuccess) {
        rc = rc ? rc : GN_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (first || ms < 0.97f * best_ms) {   // another choice must win by 3 %
        best_ms = ms;
        best = c;
      }
      first = false;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
  }
  if (h->gram_ksplit == 0 && h->gram_tile == 0) {   // only free choices go into the table
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[std::make_tuple(S, (h->Pp + TM - 1) / TM, gram_chunks(nrows))] = best;
  }
  *best_out = best;
  return GN_OK;
}
}  // namespace

int gram_split_choice(int S, int64_t Pp, int64_t nrows) {
  GramChoice ch;
  return lookup(S, Pp, nrows, &ch) ? ch.ks : 0;
}
int gram_tile_choice(int S, int64_t Pp, int64_t nrows) {
  GramChoice ch;
  return lookup(S, Pp, nrows, &ch) ? ch.tn : 0;
}

// Tune the Gram of the handle's largest row block ahead of a capture, on a zeroed operand
// (tensor-core time does not depend on the values).
int pretune_gram(gn_handle* h) {
  if (h->precision == GN_PREC_FP64 || h->gram_ksplit > 0 || h->gram_tile > 0 || h->n_rows <= 0) return GN_OK;
  const int S = h->n_slices;
  const int64_t nrows = h->jrows;
  GramChoice ks;
  if (lookup(S, h->Pp, nrows, &ks)) return GN_OK;
  const size_t opb = oz_operand_bytes(S, h->Pp, nrows);
  unsigned char* base = static_cast<unsigned char*>(h->split_ws);
  OzOperand op = oz_operand_at(base, S, h->Pp, nrows);
  if (GN_NOTE(cudaMemsetAsync(base, 0, opb, h->st)) != cudaSuccess) return GN_ERR_CUDA;
  void* part = base + opb + (size_t)CM_CHUNKS * rup(h->Pp, TM) * 8 + 256;
  return tune(h, S, op, nrows, h->G, part, &ks);
}

// Everything a step's split contractions need, allocated up front: the Gram operand of the
// largest row block, the CCF Hilbert contraction's operands (SPLIT_ALL) and the split
// factorisation's workspace and streams (SPLIT_ALL).
int prepare_for_capture(gn_handle* h) {
  if (h->precision == GN_PREC_FP64) return GN_OK;
  const int S = h->n_slices;
  size_t need = oz_operand_bytes(S, h->Pp, h->jrows) + (size_t)CM_CHUNKS * rup(h->Pp, TM) * 8 + 256 +
                gram_part_bytes(h->Pp, gram_max_split(h, h->jrows));
  if (h->precision == GN_PREC_SPLIT_ALL) {
    if (h->eq == GN_CCF && h->p.n_pts > 0) {
      const int64_t rows = h->p.n_pts < h->jrows ? h->p.n_pts : h->jrows;
      const size_t hil = oz_operand_bytes(S, rows, h->Mh) + oz_operand_bytes(S, h->Pp, h->Mh) +
                         (size_t)64 * rup(h->Pp, 128) * 8 + 512;
      if (hil > need) need = hil;
    }
    const int rc = ensure_chol_ws(h, chol_split_ws_bytes(h->Pp, S));
    if (rc) return rc;
    if (GN_NOTE(ensure_chol_streams(h)) != cudaSuccess) return GN_ERR_CUDA;
  }
  const int rc = ensure_split_ws(h, need);
  if (rc) return rc;
  return pretune_gram(h);
}

// Gram through the split GEMM: G (lower tiles) = J^T J or += (accumulate).
int split_gram(gn_handle* h, const double* J, int64_t ld, int64_t nrows, double* G, int accumulate) {
  const int S = h->n_slices;
  if (S < 1 || S > kOzMaxSlices) return GN_ERR_UNSUPPORTED;
  if (nrows <= 0) return GN_OK;
  const size_t opb = oz_operand_bytes(S, h->Pp, nrows);
  const size_t cmb = (size_t)CM_CHUNKS * rup(h->Pp, TM) * 8 + 256;
  int rc = ensure_split_ws(h, opb + cmb + gram_part_bytes(h->Pp, gram_max_split(h, nrows)));
  if (rc) return rc;
  OzOperand op = oz_operand_at(h->split_ws, S, h->Pp, nrows);
  double* part = reinterpret_cast<double*>(static_cast<unsigned char*>(h->split_ws) + opb);
  void* kpart = static_cast<unsigned char*>(h->split_ws) + opb + cmb;
  rc = oz_prepare_cols(S, J, ld, nrows, h->Pp, op, part, h->st);
  if (rc) return rc;
  // tile width and split-K factor: forced, tuned earlier for this shape, tuned now, or the defaults
  GramChoice ch;
  if (!gram_choice(h, nrows, &ch)) {
    ch.ks = h->gram_ksplit > 0 ? h->gram_ksplit : 1;
    ch.tn = h->gram_tile > 0 ? h->gram_tile : TN;
    if (!accumulate && !h->capturing && h->gram_ksplit == 0 && h->gram_tile == 0) {
      rc = tune(h, S, op, nrows, G, kpart, &ch);
      if (rc) return rc;
    }
  }
  rc = oz_gemm(S, true, op, op, h->Pp, h->Pp, G, h->Pp, accumulate ? 1 : 0, nullptr, h->flag + 2, h->st, ch.ks,
               kpart, OzRange(), ch.tn);
  if (rc) return rc;
  return GN_OK;
}

int64_t pipeline_chunk_tiles(gn_handle* h) {
  if (h->pipe_tiles == 0 || h->precision != GN_PREC_SPLIT_ALL || h->n_rows <= 0) return 0;
  if ((h->n_rows + h->jrows - 1) / h->jrows != 1) return 0;
  GramChoice ch;   // the pipeline's column chunks use square tiles without split-K
  if (!gram_choice(h, h->n_rows, &ch)) {
    ch.ks = h->gram_ksplit > 0 ? h->gram_ksplit : 1;
    ch.tn = h->gram_tile > 0 ? h->gram_tile : TN;
  }
  if (ch.ks != 1 || ch.tn != TN) return 0;
  if ((h->Pp + TM - 1) / TM < 4) return 0;   // a G this small is one strip or two
  if (h->pipe_tiles > 0) return h->pipe_tiles;
  int sms = 0;
  if (GN_NOTE(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev)) != cudaSuccess || sms < 8)
    return 0;
  return sms - sms / 8;   // leave an eighth of the SMs to the factorisation's chain
}

int split_gram_pipelined(gn_handle* h, const double* J, int64_t ld, int64_t nrows, double* G, double* A,
                         const double* gamma, int64_t chunk, cudaStream_t st, cudaStream_t sg,
                         std::vector<cudaEvent_t>& events, std::vector<cudaEvent_t>& gate) {
  const int S = h->n_slices;
  const int64_t n = h->Pp;
  if (S < 1 || S > kOzMaxSlices || nrows <= 0 || chunk <= 0) return GN_ERR_INVALID;
  const size_t opb = oz_operand_bytes(S, n, nrows);
  const size_t cmb = (size_t)CM_CHUNKS * rup(n, TM) * 8 + 256;
  int rc = ensure_split_ws(h, opb + cmb + gram_part_bytes(n, gram_max_split(h, nrows)));
  if (rc) return rc;
  OzOperand op = oz_operand_at(h->split_ws, S, n, nrows);
  double* part = reinterpret_cast<double*>(static_cast<unsigned char*>(h->split_ws) + opb);
  rc = oz_prepare_cols(S, J, ld, nrows, n, op, part, st);
  if (rc) return rc;
  auto new_event = [&](cudaEvent_t* e) -> bool {
    *e = nullptr;
    if (GN_NOTE(cudaEventCreateWithFlags(e, cudaEventDisableTiming)) != cudaSuccess) return false;
    events.push_back(*e);
    return true;
  };
  cudaEvent_t fork;
  if (!new_event(&fork) || GN_NOTE(cudaEventRecord(fork, st)) != cudaSuccess ||
      GN_NOTE(cudaStreamWaitEvent(sg, fork, 0)) != cudaSuccess)
    return GN_ERR_CUDA;
  const int64_t mt = (n + TM - 1) / TM, total = mt * (mt + 1) / 2;
  const int64_t nstrip = (n + kCholStrip - 1) / kCholStrip;
  gate.assign((size_t)nstrip, nullptr);
  auto before = [&](int64_t c) { return c * mt - c * (c - 1) / 2; };   // tiles of the columns < c
  int64_t tc = 0, strips_done = 0;
  for (int64_t t0 = 0; t0 < total; t0 += chunk) {
    OzRange rg;
    rg.tile0 = t0;
    rg.ntiles = (t0 + chunk < total) ? chunk : total - t0;
    rg.colmajor = 1;
    rc = oz_gemm(S, true, op, op, n, n, G, n, 0, nullptr, h->flag + 2, sg, 1, nullptr, rg);
    if (rc) return rc;
    while (tc < mt && before(tc + 1) <= t0 + rg.ntiles) tc++;   // tile columns [0, tc) are done
    const int64_t sd = (tc * TM >= n) ? nstrip : tc * TM / kCholStrip;   // so are strips [0, sd)
    if (sd > strips_done) {
      const int64_t c0 = strips_done * kCholStrip, c1 = (sd * kCholStrip < n) ? sd * kCholStrip : n;
      if (GN_NOTE(add_diag_band(G, A, n, n, c0, c1, gamma, sg)) != cudaSuccess) return GN_ERR_CUDA;
      cudaEvent_t e;
      if (!new_event(&e) || GN_NOTE(cudaEventRecord(e, sg)) != cudaSuccess) return GN_ERR_CUDA;
      for (int64_t t = strips_done; t < sd; t++) gate[(size_t)t] = e;
      strips_done = sd;
    }
  }
  if (strips_done != nstrip) return GN_ERR_INVALID;   // every strip must have its gate
  if (GN_NOTE(mirror_lower(G, n, n, sg)) != cudaSuccess) return GN_ERR_CUDA;
  return GN_OK;
}

}  // namespace gn

// Testing hook of the bounded waits (declared in gn.h).
extern "C" int gn_test_bounded_waits(unsigned long long wait_ns, int starve_copies) {
  gn::g_oz_wait_ns.store(wait_ns ? wait_ns : gn::kWaitNs, std::memory_order_relaxed);
  gn::g_oz_starve.store(starve_copies ? 1 : 0, std::memory_order_relaxed);
  return GN_OK;
}
