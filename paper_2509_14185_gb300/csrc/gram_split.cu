// Split-precision (Ozaki) Gram product G = J~^T J~ on the tcgen05 tensor cores.
//
// The Gauss-Newton matrix (Methods, "Second-order Optimizer") is the one truly
// dense contraction of the step.  GB300 runs BF16 on its tensor cores ~1600x
// faster than FP64, so the FP64 columns of J~ are split into BF16 slices and
// the slice products are accumulated exactly (Ozaki, Ogita, Oishi & Rump,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 2012):
//
//  1. column scale: e_j with max_i |J_ij| < 2^{e_j} (a power of two, exact);
//  2. digits: v = round(J_ij 2^{8S - e_j}) as a 64-bit integer, written as S
//     balanced base-256 digits a_1..a_S (|a_1| <= 256, |a_t| <= 128); slice t
//     holds a_t 2^{-8t}, exactly representable in BF16 (8-bit significand);
//  3. products: slice pairs (s, t) with s + t <= S + 1, grouped by level
//     l = s + t.  Within a level every product is an integer times 2^{-8l};
//     over a 128-row chunk the integer partial sums stay below 2^24, so the
//     FP32 accumulation in tensor memory is exact for levels 2, 3, 4.  Those
//     are flushed after each chunk into double-FP32 (hi, lo) registers.
//     Levels >= 5 share one accumulator over the whole K range: its FP32
//     rounding is ~2^-24 of a term that is itself <= 2^-24 of G.
//  4. G_ij = 2^{e_i + e_j} (hi + lo), written in FP64.
// Truncation error: |G_split - G|_ij <~ (S + 1) 2^{-8S} |J_:i|_2 |J_:j|_2.
//
// Kernel structure (one 128 x 128 lower-triangular output tile per CTA,
// 320 threads): warp 0 issues TMA loads of the 2 S slice tiles of each
// 32-wide K stage into a multi-stage shared-memory ring (64-byte swizzle);
// warp 1 allocates the 512 tensor-memory columns and one lane issues the
// tcgen05.mma instructions (M = N = 128, K = 16, BF16 in, FP32 accumulate);
// warps 2..9 read the accumulators with tcgen05.ld and own the double-FP32
// sums (warp w reads tensor-memory lanes 32 (w % 4) .. + 31, columns
// 64 ((w - 2) / 4) .. + 63).  Every mbarrier wait is bounded in time; a timeout
// sets bit 1 of the device status word and the CTA drains and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "gn_internal.cuh"

namespace gn {
namespace {

constexpr int TM = 128;            // output tile (rows of G)
constexpr int TN = 128;            // output tile (cols of G)
constexpr int BKS = 32;            // K per stage (64-byte rows, SWIZZLE_64B)
constexpr int KC = 128;            // exact-accumulation chunk (rows of J)
constexpr int SLICE_BYTES = TM * BKS * 2;   // one slice tile: 8 KB
constexpr int NTHREADS = 320;   // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr unsigned long long kWaitNs = 4000000000ull;   // 4 s bound on any wait
constexpr int kMaxSlices = 6;

__host__ __device__ constexpr int n_stages(int S) {
  return (2 * S * SLICE_BYTES * 4 <= 200 * 1024) ? 4 : (2 * S * SLICE_BYTES * 3 <= 200 * 1024) ? 3 : 2;
}
// The operand ring is reused at the end to park the (hi, lo) tile; the
// mbarriers live after whichever of the two is larger.
constexpr int PARK_BYTES = TM * (TN + 1) * 8;
__host__ __device__ constexpr int bar_offset(int S) {
  return n_stages(S) * 2 * S * SLICE_BYTES > PARK_BYTES ? n_stages(S) * 2 * S * SLICE_BYTES : PARK_BYTES;
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
// Bounded wait: returns false (and raises the status flag) after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* flag) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (!mbar_try(bar, parity)) {
    if (now_ns() - t0 > kWaitNs) {
      atomicOr(flag, 2);
      return false;
    }
  }
  return true;
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
// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
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

// Level of a slice pair and its tensor-memory slot: levels 2, 3, 4 -> slots 0, 1, 2; >= 5 -> 3.
__device__ __forceinline__ int slot_of(int s, int t) {
  const int l = s + t + 2;  // s, t are 0-based
  return l <= 4 ? l - 2 : 3;
}

// ---------------------------------------------------------------------------
// main kernel
// ---------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(NTHREADS, 1)
    gram_split_kernel(const __grid_constant__ CUtensorMap tmap, int64_t Ppad, int64_t Kpad, int64_t Pp,
                      const int* __restrict__ ecol, double* G, int64_t ldg, int accumulate, int* flag) {
  constexpr int NST = n_stages(S);
  constexpr int STAGE_BYTES = 2 * S * SLICE_BYTES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + bar_offset(S));
  uint64_t* empty = full + NST;
  uint64_t* acc_full = empty + NST;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* done = acc_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int abort_cta;
  __shared__ int ecs[2][TM];   // column exponents of this tile's rows (0) and columns (1)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // lower-triangular tile (ti >= tj) of this CTA
  const int64_t t = blockIdx.x;
  int64_t ti = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= t) ti++;
  while (ti * (ti + 1) / 2 > t) ti--;
  const int64_t tj = t - ti * (ti + 1) / 2;
  const int nk = (int)(Kpad / BKS);
  const int nchunk = (int)(Kpad / KC);
  constexpr int SPC = KC / BKS;  // stages per chunk

  if (threadIdx.x == 0) {
    abort_cta = 0;
    for (int i = 0; i < NST; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 8);
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      const int rowA = (int)(ti * TM), rowB = (int)(tj * TN);
      int issued = 0;
      for (int kt = 0; kt < nk; kt++) {
        const int st = kt % NST;
        if (kt >= NST) {
          if (!mbar_wait(&empty[st], ((kt / NST) - 1) & 1, flag)) {
            abort_cta = 1;
            break;
          }
        }
        if (*(volatile int*)&abort_cta) break;
        unsigned char* base = smem + st * STAGE_BYTES;
        mbar_expect_tx(&full[st], STAGE_BYTES);
#pragma unroll
        for (int s = 0; s < S; s++) {
          tma_load_2d(base + s * SLICE_BYTES, &tmap, kt * BKS, (int)(s * Ppad) + rowA, &full[st]);
          tma_load_2d(base + (S + s) * SLICE_BYTES, &tmap, kt * BKS, (int)(s * Ppad) + rowB, &full[st]);
        }
        issued = kt + 1;
      }
      // drain: every issued stage must land before the CTA may exit
      for (int kt = (issued > NST ? issued - NST : 0); kt < issued; kt++) mbar_wait(&full[kt % NST], (kt / NST) & 1, flag);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      for (int c = 0; c < nchunk && ok; c++) {
        for (int q = 0; q < SPC && ok; q++) {
          const int kt = c * SPC + q;
          const int st = kt % NST;
          if (!mbar_wait(&full[st], (kt / NST) & 1, flag)) { ok = false; break; }
          if (q == 0 && c > 0) {
            // head accumulators must have been read before they are reset
            if (!mbar_wait(acc_empty, (c - 1) & 1, flag)) { ok = false; break; }
          }
          tc_fence_after();
          const uint32_t base = smem_u32(smem + st * STAGE_BYTES);
#pragma unroll
          for (int s = 0; s < S; s++)
#pragma unroll
            for (int u = 0; u < S; u++) {
              if (s + u > S - 1) continue;  // keep levels s + t <= S + 1 (1-based)
              const int slot = slot_of(s, u);
#pragma unroll
              for (int kk = 0; kk < BKS / 16; kk++) {
                const uint64_t da = smem_desc(base + s * SLICE_BYTES + kk * 32);
                const uint64_t db = smem_desc(base + (S + u) * SLICE_BYTES + kk * 32);
                // first contribution of this slot in the chunk (head) or in the whole run (tail) resets it
                bool first;
                if (slot < 3) {
                  // first pair of this level within the chunk: smallest s with s + u fixed
                  const int lvl = s + u;
                  const int s_first = 0;
                  first = (q == 0 && kk == 0 && s == s_first && u == lvl - s_first);
                } else {
                  first = (kt == 0 && kk == 0 && s == 0 && u == 3);
                }
                mma_bf16(tmem + slot * TN, da, db, first ? 0u : 1u);
              }
            }
          mma_commit(&empty[st]);
        }
        if (ok) mma_commit(acc_full);
      }
      if (!ok) abort_cta = 1;
      // every issued MMA must complete before tensor memory is released
      mma_commit(done);
      mbar_wait(done, 0, flag);
    }
  } else {
    // ---------------- epilogue: 8 warps, 64 columns each ----------------
    constexpr int EC = 64;                      // columns per epilogue thread
    const int quad = warp & 3;
    const int qcol = (warp - 2) >> 2;          // column half 0..1
    const int row = quad * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(qcol * EC);
    {
      // stage the tile's column exponents (Ppad-padded, so always in range)
      ecs[qcol][row] = ecol[(qcol == 0 ? ti * TM : tj * TN) + row];
      asm volatile("bar.sync 1, 256;" ::: "memory");   // the 8 epilogue warps only
    }
    float hi[EC], lo[EC];
#pragma unroll
    for (int i = 0; i < EC; i++) { hi[i] = 0.f; lo[i] = 0.f; }
    constexpr int nhead = S < 3 ? S : 3;        // head levels present: 2..min(S+1, 4)
    bool ok = true;
    for (int c = 0; c < nchunk; c++) {
      if (!mbar_wait(acc_full, c & 1, flag)) { ok = false; break; }
      tc_fence_after();
#pragma unroll
      for (int slot = 0; slot < nhead; slot++) {
#pragma unroll
        for (int part = 0; part < EC / 16; part++) {
          float v[16];
          tmem_ld16(lane_base + (uint32_t)(slot * TN + part * 16), v);
#pragma unroll
          for (int i = 0; i < 16; i++) dd_add(hi[part * 16 + i], lo[part * 16 + i], v[i]);
        }
      }
      if (S >= 4 && c == nchunk - 1) {
#pragma unroll
        for (int part = 0; part < EC / 16; part++) {
          float v[16];
          tmem_ld16(lane_base + (uint32_t)(3 * TN + part * 16), v);
#pragma unroll
          for (int i = 0; i < 16; i++) dd_add(hi[part * 16 + i], lo[part * 16 + i], v[i]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
    }
    // All loads have landed and all MMAs have completed (the last acc_full),
    // so the operand ring is free: park (hi, lo) there, then convert and store
    // the tile with coalesced writes.
    float2* park = reinterpret_cast<float2*>(smem);
    if (ok) {
#pragma unroll
      for (int i = 0; i < EC; i++) park[row * (TN + 1) + qcol * EC + i] = make_float2(hi[i], lo[i]);
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (ok) {
      const int et = (warp - 2) * 32 + lane;
      for (int idx = et; idx < TM * TN; idx += 256) {
        const int r = idx / TN, cc = idx % TN;
        const int64_t gi = ti * TM + r, gj = tj * TN + cc;
        if (gi < Pp && gj < Pp) {
          const float2 hl = park[r * (TN + 1) + cc];
          double v = ((double)hl.x + (double)hl.y) * pow2(ecs[0][r]) * pow2(ecs[1][cc]);
          if (accumulate) v += G[gi * ldg + gj];
          G[gi * ldg + gj] = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// ---------------------------------------------------------------------------
// pre-pass: column exponents and the slice split (transposed, K-major)
// ---------------------------------------------------------------------------
constexpr int CM_CHUNKS = 64;
__global__ void colmax_partial(const double* __restrict__ J, int64_t ld, int64_t nrows, int64_t ncols, double* part) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  const int c = blockIdx.y;
  const int64_t per = (nrows + CM_CHUNKS - 1) / CM_CHUNKS;
  const int64_t r0 = c * per, r1 = (r0 + per < nrows) ? r0 + per : nrows;
  double m = 0.0;
  for (int64_t r = r0; r < r1; r++) m = fmax(m, fabs(J[r * ld + j]));
  part[(int64_t)c * ncols + j] = m;
}
__global__ void colexp_kernel(const double* __restrict__ part, int64_t ncols, int64_t Ppad, int* ecol) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Ppad) return;
  int e = 0;
  if (j < ncols) {
    double m = 0.0;
    for (int c = 0; c < CM_CHUNKS; c++) m = fmax(m, part[(int64_t)c * ncols + j]);
    if (m > 0.0 && isfinite(m)) frexp(m, &e);  // m = f 2^e, f in [0.5, 1): 2^e > m
  }
  ecol[j] = e;
}

// 64 rows x 32 columns of J per block -> S slice rows of 64 BF16 each (per column).
template <int S>
__global__ void __launch_bounds__(256) split_kernel(const double* __restrict__ J, int64_t ld, int64_t nrows,
                                                    int64_t ncols, const int* __restrict__ ecol, int64_t Ppad,
                                                    int64_t Kpad, __nv_bfloat16* out) {
  __shared__ __align__(16) __nv_bfloat16 sl[S][32][64 + 8];
  const int t = threadIdx.x;
  const int64_t k0 = (int64_t)blockIdx.x * 64, j0 = (int64_t)blockIdx.y * 32;
  const int jj = t & 31;
  const int64_t j = j0 + jj;
  const int e = (j < Ppad) ? ecol[j] : 0;
#pragma unroll
  for (int r = 0; r < 8; r++) {
    const int kk = (t >> 5) + 8 * r;
    const int64_t k = k0 + kk;
    double x = (k < nrows && j < ncols) ? J[k * ld + j] : 0.0;
    long long v = llrint(ldexp(x, 8 * S - e));
    int a[S];
#pragma unroll
    for (int q = S - 1; q >= 1; q--) {
      const long long d = (v + 128) >> 8;
      a[q] = (int)(v - (d << 8));
      v = d;
    }
    a[0] = (int)v;
#pragma unroll
    for (int q = 0; q < S; q++) sl[q][jj][kk] = __float2bfloat16_rn(ldexpf((float)a[q], -8 * (q + 1)));
  }
  __syncthreads();
  // write: per (slice, column) 64 BF16 = 128 bytes, 16 bytes per thread
  for (int idx = t; idx < S * 32 * 8; idx += 256) {
    const int q = idx / (32 * 8), rem = idx % (32 * 8);
    const int c = rem / 8, seg = rem % 8;
    const int64_t col = j0 + c;
    if (col >= Ppad || k0 + seg * 8 >= Kpad) continue;
    const uint4 val = *reinterpret_cast<const uint4*>(&sl[q][c][seg * 8]);
    *reinterpret_cast<uint4*>(out + ((int64_t)q * Ppad + col) * Kpad + k0 + seg * 8) = val;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

struct SplitWs {
  int64_t Ppad, Kpad;
  int S;
  __nv_bfloat16* slices;
  int* ecol;
  double* part;
  size_t bytes;
};

template <int S>
int launch_split(gn_handle* h, const double* J, int64_t ld, int64_t nrows, double* G, int accumulate, SplitWs& ws) {
  cudaStream_t st = h->st;
  const int64_t Pp = h->Pp;
  // pre-pass
  {
    dim3 g((unsigned)((Pp + 127) / 128), CM_CHUNKS);
    colmax_partial<<<g, 128, 0, st>>>(J, ld, nrows, Pp, ws.part);
    count_launch();
    colexp_kernel<<<(unsigned)((ws.Ppad + 255) / 256), 256, 0, st>>>(ws.part, Pp, ws.Ppad, ws.ecol);
    count_launch();
    dim3 gs((unsigned)(ws.Kpad / 64), (unsigned)(ws.Ppad / 32));
    split_kernel<S><<<gs, 256, 0, st>>>(J, ld, nrows, Pp, ws.ecol, ws.Ppad, ws.Kpad, ws.slices);
    count_launch();
  }
  if (GN_NOTE(cudaGetLastError()) != cudaSuccess) return GN_ERR_CUDA;
  EncodeTiledFn enc = get_encode();
  if (!enc) {
    set_detail(__FILE__, __LINE__, "cuTensorMapEncodeTiled entry point not found");
    return GN_ERR_UNSUPPORTED;
  }
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  cuuint64_t dims[2] = {(cuuint64_t)ws.Kpad, (cuuint64_t)(S * ws.Ppad)};
  cuuint64_t strides[1] = {(cuuint64_t)(ws.Kpad * 2)};
  cuuint32_t box[2] = {BKS, TM};
  cuuint32_t estr[2] = {1, 1};
  CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ws.slices, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    char msg[64];
    snprintf(msg, sizeof(msg), "cuTensorMapEncodeTiled returned %d", (int)cr);
    set_detail(__FILE__, __LINE__, msg);
    return GN_ERR_CUDA;
  }
  constexpr int NST = n_stages(S);
  const size_t smem = (size_t)bar_offset(S) + 1024 + 256;
  if (GN_NOTE(cudaFuncSetAttribute(gram_split_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return GN_ERR_CUDA;
  const int64_t nt = ws.Ppad / TM;
  const int64_t tiles = nt * (nt + 1) / 2;
  if (GN_NOTE(cudaMemsetAsync(h->flag + 2, 0, sizeof(int), st)) != cudaSuccess) return GN_ERR_CUDA;
  gram_split_kernel<S><<<(unsigned)tiles, NTHREADS, smem, st>>>(map, ws.Ppad, ws.Kpad, Pp, ws.ecol, G, Pp,
                                                                 accumulate, h->flag + 2);
  count_launch();
  if (GN_NOTE(cudaGetLastError()) != cudaSuccess) return GN_ERR_CUDA;
  int hflag = 0;
  if (GN_NOTE(cudaMemcpyAsync(&h->hpin[9], h->flag + 2, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      GN_NOTE(cudaStreamSynchronize(st)) != cudaSuccess)
    return GN_ERR_CUDA;
  memcpy(&hflag, &h->hpin[9], sizeof(int));
  if (hflag & 2) return GN_ERR_TIMEOUT;
  return GN_OK;
}

}  // namespace

int split_gram(gn_handle* h, const double* J, int64_t ld, int64_t nrows, double* G, int accumulate) {
  const int S = h->n_slices;
  if (S < 1 || S > kMaxSlices) return GN_ERR_UNSUPPORTED;
  if (nrows <= 0) return GN_OK;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, h->dev);
  if (major != 10) return GN_ERR_UNSUPPORTED;
  SplitWs ws;
  ws.S = S;
  ws.Ppad = (h->Pp + TM - 1) / TM * TM;
  ws.Kpad = (nrows + KC - 1) / KC * KC;
  const size_t slice_bytes = (size_t)S * ws.Ppad * ws.Kpad * 2;
  const size_t need = slice_bytes + (size_t)ws.Ppad * sizeof(int) + (size_t)CM_CHUNKS * ws.Ppad * 8 + 4096;
  if (h->split_ws_bytes < need) {
    if (h->split_ws) cudaFree(h->split_ws);
    h->split_ws = nullptr;
    h->split_ws_bytes = 0;
    if (cudaMalloc(&h->split_ws, need) != cudaSuccess) return GN_ERR_OOM;
    h->split_ws_bytes = need;
  }
  unsigned char* p = static_cast<unsigned char*>(h->split_ws);
  ws.slices = reinterpret_cast<__nv_bfloat16*>(p);
  ws.part = reinterpret_cast<double*>(p + ((slice_bytes + 255) / 256) * 256);
  ws.ecol = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(ws.part) + (size_t)CM_CHUNKS * ws.Ppad * 8);
  switch (S) {
    case 1: return launch_split<1>(h, J, ld, nrows, G, accumulate, ws);
    case 2: return launch_split<2>(h, J, ld, nrows, G, accumulate, ws);
    case 3: return launch_split<3>(h, J, ld, nrows, G, accumulate, ws);
    case 4: return launch_split<4>(h, J, ld, nrows, G, accumulate, ws);
    case 5: return launch_split<5>(h, J, ld, nrows, G, accumulate, ws);
    default: return launch_split<6>(h, J, ld, nrows, G, accumulate, ws);
  }
}

}  // namespace gn
