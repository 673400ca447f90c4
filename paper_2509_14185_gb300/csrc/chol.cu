// Damped FP64 Cholesky solve (G + gamma I) delta = g of the Gauss-Newton step
// (Methods, "Second-order Optimizer").
//
// Blocked right-looking factorisation on a row-major matrix, lower triangle,
// block size 64:
//   1. one CTA factors the 64 x 64 diagonal block in shared memory and forms
//      its inverse Linv_k in the same sweep (kept for the panel and the
//      triangular solves);
//   2. the panel below it is solved on the CUDA cores, L21 = A21 Linv_k^T
//      (FP64), and on the split path the same kernel writes L21's BF16 slices
//      for the trailing update;
//   3. the trailing matrix is updated A22 -= L21 L21^T (lower tiles only).
// A non-positive pivot sets a device flag; later blocks skip their work and
// the host escalates the damping.  The triangular solves use the stored
// diagonal inverses: a tiny 64 x 64 product per block plus a GEMV of the
// remaining vector spread over all SMs.
#include <cmath>
#include <type_traits>
#include <vector>

#include "gn_internal.cuh"

namespace gn {
namespace {

constexpr int NB = kCholNB;

// 2^e (exact) for the exponent range of a scaled block, ldexp outside it
__device__ __forceinline__ double p2(int e) {
  return (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52) : ldexp(1.0, e);
}
__device__ __forceinline__ float p2f(int e) {   // e in [-126, 127]
  return __int_as_float((e + 127) << 23);
}

// Arithmetic of the diagonal-block factor.  Arith64 is plain FP64.  ArithDF
// carries each value as an unevaluated sum of two floats (hi + lo, about 48
// significant bits) on the FP32 pipe: the sweep is a chain of 64 dependent
// steps, and GB300's FP64 units are both narrow (about 1/60 of the FP32 rate)
// and long-latency, so the FP32 pipe runs it several times faster.  Each also
// provides the scaled load (A - U) 2^k, the scaled store v 2^k and 1/sqrt(d).
struct Arith64 {
  using T = double;
  static __device__ __forceinline__ T one() { return 1.0; }
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ bool positive(T d) { return d > 0.0 && isfinite(d); }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T fnma(T s, T a, T b) { return fma(-a, b, s); }   // s - a b
  static __device__ __forceinline__ T rcp(T d) { return 1.0 / d; }
  static __device__ __forceinline__ T rsqrt(T d) { return 1.0 / sqrt(d); }
  static __device__ __forceinline__ T load_scaled(double a, const float2* u, int k) {
    if (u) a -= (double)u->x + (double)u->y;
    return a * p2(k);
  }
  static __device__ __forceinline__ double store_scaled(T v, int k) { return v * p2(k); }
};

struct DF {
  float h, l;
};

// a 2^k as a double-float pair, by integer operations on the bits (no FP64
// arithmetic): the top 24 significand bits form hi exactly, the low 29 bits
// rounded to 24 form lo.  Returns false (caller falls back) for zero-exponent
// or non-finite a and for results outside [2^-70, 2^127).
__device__ __forceinline__ bool df_split_scaled(double a, int k, float& h, float& l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  if ((b << 1) == 0ull) {
    h = l = 0.f;
    return true;
  }
  const int ex = (int)((b >> 52) & 0x7ff);
  const int e = ex - 1023 + k;
  if (ex == 0 || ex == 0x7ff || e < -70 || e > 126) return false;
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  h = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | ((unsigned)(mant >> 29) & 0x7fffffu));
  const float lo = __fmul_rn(__uint2float_rn((unsigned)(mant & ((1u << 29) - 1))), p2f(e - 52));
  l = sign ? -lo : lo;
  return true;
}
// x 2^k as a double, by integer operations (exact for normal x and a normal result)
__device__ __forceinline__ double f2d_scaled(float x, int k) {
  const unsigned b = __float_as_uint(x);
  const int ex = (int)((b >> 23) & 0xff);
  if (ex == 0 || ex == 0xff) return (double)x * p2(k);   // zero, subnormal or non-finite: FP64 path
  const int e = ex - 127 + k + 1023;
  if (e <= 0 || e >= 2047) return (double)x * p2(k);
  return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) |
                                          ((unsigned long long)e << 52) |
                                          ((unsigned long long)(b & 0x7fffffu) << 29)));
}

struct ArithDF {
  using T = DF;
  static __device__ __forceinline__ T from(double a) {
    const float h = __double2float_rn(a);
    return {h, __double2float_rn(a - (double)h)};
  }
  static __device__ __forceinline__ T one() { return {1.f, 0.f}; }
  static __device__ __forceinline__ T zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ bool positive(T d) { return d.h > 0.f && isfinite(d.h); }
  // a + b (TwoSum of the high parts, low parts added, Fast2Sum renormalisation)
  static __device__ __forceinline__ T add(T a, T b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    const float t = __fadd_rn(err, __fadd_rn(a.l, b.l));
    const float hi = __fadd_rn(s, t);
    return {hi, __fsub_rn(t, __fsub_rn(hi, s))};
  }
  // a b: exact product of the high parts (FMA) plus the cross terms, renormalised (Fast2Sum)
  static __device__ __forceinline__ T mul(T a, T b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    const float hi = __fadd_rn(p, e);
    return {hi, __fsub_rn(e, __fsub_rn(hi, p))};
  }
  // s - a b: the product as above, its high part subtracted exactly (TwoSum)
  static __device__ __forceinline__ T fnma(T s, T a, T b) {
    const float p = __fmul_rn(a.h, b.h);
    float pe = __fmaf_rn(a.h, b.h, -p);
    pe = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, pe));
    const float d = __fsub_rn(s.h, p);
    const float bb = __fsub_rn(d, s.h);
    const float err = __fadd_rn(__fsub_rn(s.h, __fsub_rn(d, bb)), __fsub_rn(-p, bb));
    const float t = __fadd_rn(err, __fsub_rn(s.l, pe));
    const float hi = __fadd_rn(d, t);
    return {hi, __fsub_rn(t, __fsub_rn(hi, d))};
  }
  // s - a b for a running sum: as fnma, but the low part only collects the rounding errors (no
  // renormalisation per term; a few dozen terms keep it far below the high part), so a sum of
  // products costs 12 FP32 operations per term instead of 15.  add() renormalises at the end.
  static __device__ __forceinline__ T fnma_lazy(T s, T a, T b) {
    const float p = __fmul_rn(a.h, b.h);
    float pe = __fmaf_rn(a.h, b.h, -p);
    pe = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, pe));
    const float d = __fsub_rn(s.h, p);
    const float bb = __fsub_rn(d, s.h);
    const float err = __fadd_rn(__fsub_rn(s.h, __fsub_rn(d, bb)), __fsub_rn(-p, bb));
    return {d, __fadd_rn(s.l, __fsub_rn(err, pe))};
  }
  // 1 / d: the FP32 reciprocal r and one Newton correction r (1 - d r) kept as the low part
  static __device__ __forceinline__ T rcp(T d) {
    const float r = __frcp_rn(d.h);
    float e = __fmaf_rn(-d.h, r, 1.0f);
    e = __fmaf_rn(-d.l, r, e);
    const float c = __fmul_rn(r, e);
    const float hi = __fadd_rn(r, c);
    return {hi, __fsub_rn(c, __fsub_rn(hi, r))};
  }
  // 1 / sqrt(d): FP32 estimate, then two Newton steps r += r (1 - d r^2) / 2 in double-float
  static __device__ __forceinline__ T rsqrt(T d) {
    T r = {rsqrtf(d.h), 0.f};
#pragma unroll
    for (int it = 0; it < 2; it++) {
      const T e = add(one(), mul({-d.h, -d.l}, mul(r, r)));   // 1 - d r^2
      r = add(r, mul(r, {0.5f * e.h, 0.5f * e.l}));
    }
    return r;
  }
  static __device__ __forceinline__ T load_scaled(double a, const float2* u, int k) {
    float h, l;
    if (!df_split_scaled(a, k, h, l) || (u && (k < -126 || k > 127))) {
      if (u) a -= (double)u->x + (double)u->y;   // out of the fast path's range: FP64
      return from(a * p2(k));
    }
    T v = {h, l};
    if (u) {
      const float s = p2f(k);   // exact power-of-two scaling of U's pair
      v = add(v, {-__fmul_rn(u->x, s), -__fmul_rn(u->y, s)});
    }
    return v;
  }
  static __device__ __forceinline__ double store_scaled(T v, int k) { return f2d_scaled(v.h, k) + f2d_scaled(v.l, k); }
};

constexpr int kPotrfTPR = 16;                       // threads per row of the diagonal block
constexpr size_t kPotrfSmem = (size_t)(NB * (NB + 1) + 4 * NB) * 8;   // final columns + 2 x 2 broadcast rows

// Factor and invert the diagonal block B = A[k0:k0+kb, k0:k0+kb] (minus U, the
// double-FP32 sum of earlier trailing updates, when U is given).
//
// B is first scaled symmetrically by powers of two, B' = D B D with
// D_ii = 2^-sc[i] and B'_ii in [1, 4), so every value stays O(1) (exact; it
// also keeps the double-float variant inside FP32's exponent range).  The
// sweep is the LDL^T form of right-looking elimination: at column j every row
// i > j applies, with d_j = S[j][j] and a_i = S[i][j] / d_j,
//     S[i][c] -= a_i S[c][j]    (j < c <= i: the trailing block)
//     Y[i][c] -= a_i Y[j][c]    (c <= j: the inverse, Y = I at the start)
// so no value is rescaled inside the chain.  S[i][c] and Y[i][c] share one
// register: column c of S is final (and published) at step c, exactly when
// Y[i][c] starts to accumulate.  Thread (i, g) holds row i's elements
// c = g + TPR m (m < 64 / TPR) in registers: independent chains per thread,
// and with TPR = 16 (1024 threads, 4 chains each) 32 warps to hide the FP32
// latency of the double-float arithmetic.  The sweep is a chain of dependent
// steps: fewer threads per row (8: 5 % slower, 4: 30 % slower on GB300) leave
// that latency exposed, though each thread then repeats less per-row work.
// Each step publishes column j of S and row j of Y to shared memory (double
// buffered, so one barrier per column suffices).  At the end
// L'[i][j] = S[i][j] / sqrt(d_j) and L'^{-1}[i][c] = Y[i][c] / sqrt(d_i);
// undoing D gives L = D^-1 L' and Linv = L'^{-1} D, written in FP64.
template <class AR, int TPR>
__global__ void __launch_bounds__(NB * TPR) potrf_inv_kernel(double* A, int64_t lda, int64_t k0, int kb,
                                                                  const float2* __restrict__ U, int64_t ldu,
                                                                  double* Linv, float2* LinvDF, int* scOut,
                                                                  const double* fw, double* fy, float2* fyDF,
                                                                  int* flag) {
  using T = typename AR::T;
  constexpr int EPT = NB / TPR;   // elements (columns) per thread
  extern __shared__ __align__(16) unsigned char smraw[];
  T (*Lf)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(smraw);   // unscaled final columns S[i][j], i >= j
  T* colbuf = reinterpret_cast<T*>(smraw) + NB * (NB + 1);     // [2][NB]: column j of S
  T* rowbuf = colbuf + 2 * NB;                                 // [2][NB]: row j of Y; reused for 1/sqrt(d)
  __shared__ int sc[NB];
  if (*flag) return;
  const int t = threadIdx.x, i = t / TPR, g = t % TPR;
  if (t < NB) {
    int e = 0;
    if (t < kb) {
      double d = A[(k0 + t) * lda + k0 + t];
      if (U) {
        const float2 u = U[(k0 + t) * ldu + k0 + t];
        d -= (double)u.x + (double)u.y;
      }
      if (d > 0.0 && isfinite(d)) e = ilogb(d) >> 1;   // floor(log2(d) / 2)
    }
    sc[t] = e;
  }
  __syncthreads();
  T X[EPT];
#pragma unroll
  for (int m = 0; m < EPT; m++) {
    const int c = g + TPR * m;
    X[m] = AR::zero();
    if (i < kb && c <= i) {
      float2 u;
      if (U) u = U[(k0 + i) * ldu + k0 + c];
      X[m] = AR::load_scaled(A[(k0 + i) * lda + k0 + c], U ? &u : nullptr, -(sc[i] + sc[c]));
    }
  }
  bool bad = false;
  for (int j = 0; j < kb; j++) {
    T* cb = colbuf + (j & 1) * NB;
    T* rb = rowbuf + (j & 1) * NB;
    if (i < kb) {
      if (g == j % TPR && i >= j) {
        // the owner of column j: constant register indices only (no indexed registers)
        const int jm = j / TPR;
        T v = AR::zero();
#pragma unroll
        for (int m = 0; m < EPT; m++)
          if (m == jm) {
            v = X[m];
            X[m] = AR::zero();
          }
        // from here on the register accumulates Y[i][j] (0 below the diagonal of I)
        cb[i] = v;
        Lf[i][j] = v;
      }
      if (i == j) {
#pragma unroll
        for (int m = 0; m < EPT; m++)
          if (g + TPR * m < j) rb[g + TPR * m] = X[m];
      }
    }
    __syncthreads();
    const T d = cb[j];
    if (!AR::positive(d)) {   // every thread reads the same pivot: the exit is uniform
      bad = true;
      break;
    }
    if (i > j && i < kb) {
      const T a = AR::mul(cb[i], AR::rcp(d));
      const int mmax = (i - g) >= 0 ? (i - g) / TPR : -1;   // columns c = g + TPR m <= i
#pragma unroll
      for (int m = 0; m < EPT; m++) {
        if (m > mmax) break;
        const int c = g + TPR * m;
        // trailing: S[c][j] (column j); inverse: Y[j][c] (row j), with Y[j][j] = 1
        const T* src = (c > j) ? &cb[c] : &rb[c];
        const T v = (c == j) ? AR::one() : *src;
        X[m] = AR::fnma(X[m], a, v);
      }
    }
  }
  if (bad) {
    if (t == 0) atomicExch(flag, 1);
    return;
  }
  __syncthreads();
  T* rs = rowbuf;   // 1/sqrt(d_j)
  if (t < kb) rs[t] = AR::rsqrt(Lf[t][t]);
  __syncthreads();
  double* Lk = Linv + (k0 / NB) * NB * NB;
  float2* Lf2 = LinvDF ? LinvDF + (k0 / NB) * NB * NB : nullptr;
#pragma unroll
  for (int m = 0; m < EPT; m++) {
    const int c = g + TPR * m;
    T v = AR::zero();
    if (i < kb && c <= i) v = (c == i) ? rs[i] : AR::mul(X[m], rs[i]);   // L'^{-1}[i][c] = Y[i][c] / sqrt(d_i)
    Lk[i * NB + c] = (i < kb && c <= i) ? AR::store_scaled(v, -sc[c]) : 0.0;
    if constexpr (std::is_same<T, DF>::value) {
      if (Lf2) Lf2[i * NB + c] = make_float2(v.h, v.l);   // for the double-float panel solve (without D)
    }
  }
  if (Lf2 && t < NB) scOut[(k0 / NB) * NB + t] = sc[t];
  if constexpr (std::is_same<T, DF>::value) {
    // forward substitution, block k: y_k = Linv_k w_k = L'^{-1} (D w_k); thread (i, g) sums its
    // columns, the TPR threads of row i (consecutive lanes) combine their sums
    if (fw) {
      T acc = AR::zero();
#pragma unroll
      for (int m = 0; m < EPT; m++) {
        const int c = g + TPR * m;
        if (i < kb && c <= i) {
          const T v = (c == i) ? rs[i] : AR::mul(X[m], rs[i]);
          acc = AR::add(acc, AR::mul(v, AR::load_scaled(fw[k0 + c], nullptr, -sc[c])));
        }
      }
#pragma unroll
      for (int o = 1; o < TPR; o <<= 1) {
        const T other = {__shfl_xor_sync(0xffffffffu, acc.h, o), __shfl_xor_sync(0xffffffffu, acc.l, o)};
        acc = AR::add(acc, other);
      }
      if (g == 0 && i < kb) {
        fy[k0 + i] = AR::store_scaled(acc, 0);
        fyDF[i] = make_float2(acc.h, acc.l);
      }
    }
  }
  for (int idx = t; idx < NB * NB; idx += blockDim.x) {
    const int r = idx / NB, c = idx % NB;
    if (r < kb && c <= r) A[(k0 + r) * lda + k0 + c] = AR::store_scaled(AR::mul(Lf[r][c], rs[c]), sc[r]);
  }
}

// Blocked double-float factor of the diagonal block (the split path's critical-path kernel).
// B = A[k0:k0+kb, k0:k0+kb] - U (lower), scaled B' = D B D by powers of two (D_ii = 2^-sc[i],
// B'_ii in [1, 4)), factored as B' = L' L'^T with L'^{-1} formed alongside.  Writes only
// double-float results: L' (LDF), L'^{-1} (LinvDF), the scales, and (with fw) the
// forward-substitution block y_k = L'^{-1} D w_k.  The FP64 copies the triangular solves read
// (L = D^-1 L' into A, Linv = L'^{-1} D) are formed for all blocks at once after the chain
// (diag_to_fp64_kernel): their FP64 additions (two per element; GB300's FP64 pipe retires
// about two per clock per SM) took a tenth of this kernel's time.  Rows and columns kb .. 63
// are padded with the identity.
//
// The same LDL^T elimination as potrf_inv_kernel (S: unscaled columns L_unit D; Y = L_unit^{-1}),
// reordered into four 16-column sub-panels p so that only a 16-step chain is latency-bound:
//  (a) 256 threads (one element each) sweep the 16 x 16 diagonal sub-block column by column
//      (S and Y_pp = its unit-lower inverse share registers, as in the unblocked kernel; the
//      pivots' reciprocals are kept);
//  (b) every thread then forms, into registers: the sub-panel rows below, S21 = B21 Y_pp^T,
//      with T21 = S21 diag(1/d); and the sub-panel's own Y rows for the earlier columns,
//      Y_p,<c0 <- Y_pp Y_p,<c0 (the rows' share of the elimination within the sub-panel);
//  (c) the trailing rank-16 update of the rows below: S22 -= T21 S21^T on the lower triangle,
//      and Y_below -= T21 Y_p on the columns < c0 + 16.  Only the next sub-panel's diagonal
//      block is updated before the next sweep; the rest runs on the other 768 threads beside
//      that sweep (it touches neither the block nor the sweep's buffers).
// Each product is the same double-float arithmetic (about 48 significant bits) as the
// unblocked sweep; only the order of the updates changes.  1024 threads, one CTA: the
// phases (b) and (c) give most threads one or two outputs, each a 16-term double-float dot
// product summed in two interleaved partial sums (two dependent chains of 8).
constexpr int kPbThreads = 1024;
constexpr int kPbB = 16;                       // sub-panel width
constexpr int kPbLd = NB + 1;                  // row stride of the shared S and Y (DF elements)
constexpr size_t kPbSmem = (size_t)(2 * NB * kPbLd + (NB - kPbB) * kPbB + 4 * kPbB + 2 * NB) * sizeof(DF) +
                           (size_t)(NB + 4) * sizeof(int);

__global__ void __launch_bounds__(kPbThreads) potrf_blk_kernel(const double* A, int64_t lda, int64_t k0, int kb,
                                                               const float2* __restrict__ U, int64_t ldu,
                                                               float2* LDF, float2* LinvDF, int* scOut,
                                                               const double* fw, double* fy, float2* fyDF,
                                                               int* flag) {
  using AR = ArithDF;
  using T = DF;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Sm = reinterpret_cast<T*>(smraw);                 // [NB][kPbLd] S (lower, diagonal included)
  T* Ym = Sm + NB * kPbLd;                             // [NB][kPbLd] Y (lower, unit diagonal)
  T* Tm = Ym + NB * kPbLd;                             // [NB - 16][16] T21 of the current sub-panel
  T* colbuf = Tm + (NB - kPbB) * kPbB;                 // [2][16] the sweep's column j of S
  T* rowbuf = colbuf + 2 * kPbB;                       // [2][16] the sweep's row j of Y
  T* rd = rowbuf + 2 * kPbB;                           // [NB] 1 / d_j
  T* rsd = rd + NB;                                    // [NB] 1 / sqrt(d_j)
  int* sc = reinterpret_cast<int*>(rsd + NB);          // [NB] scales
  int* bad = sc + NB;
  auto S = [&](int i, int c) -> T& { return Sm[i * kPbLd + c]; };
  auto Y = [&](int i, int c) -> T& { return Ym[i * kPbLd + c]; };
  if (*flag) return;
  const int t = threadIdx.x;
  if (t < NB) {
    int e = 0;
    if (t < kb) {
      double d = A[(k0 + t) * lda + k0 + t];
      if (U) {
        const float2 u = U[(k0 + t) * ldu + k0 + t];
        d -= (double)u.x + (double)u.y;
      }
      if (d > 0.0 && isfinite(d)) e = ilogb(d) >> 1;   // floor(log2(d) / 2)
    }
    sc[t] = e;
  }
  if (t == 0) *bad = 0;
  // load S = D (A - U) D on the lower triangle (identity on the padding), Y = I; the block's
  // global loads are all issued before the scales are known
  constexpr int kPer = NB * NB / kPbThreads;
  double av[kPer];
  float2 uv[kPer];
#pragma unroll
  for (int m = 0; m < kPer; m++) {
    const int idx = t + m * kPbThreads, i = idx / NB, c = idx % NB;
    const bool in = c <= i && i < kb;
    av[m] = in ? A[(k0 + i) * lda + k0 + c] : 0.0;
    uv[m] = (in && U) ? U[(k0 + i) * ldu + k0 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < kPer; m++) {
    const int idx = t + m * kPbThreads, i = idx / NB, c = idx % NB;
    if (c > i) continue;
    T v = (i == c) ? AR::one() : AR::zero();
    if (i < kb) {
      const float2 u = uv[m];
      v = AR::load_scaled(av[m], U ? &u : nullptr, -(sc[i] + sc[c]));
    }
    S(i, c) = v;
    Y(i, c) = (i == c) ? AR::one() : AR::zero();
  }
  __syncthreads();

  // Output o of sub-panel c0's trailing rank-16 update (phase (c)): o < nS indexes the lower
  // triangle of S22 (rows and columns from c0 + 16, row by row, so the first 136 outputs are the
  // next sub-panel's diagonal block), the rest Y_below[:, < c0 + 16] row by row.
  auto trailing = [&](int c0, int o) {
    const int nb_rows = NB - c0 - kPbB, cw = c0 + kPbB;
    const int nS = nb_rows * (nb_rows + 1) / 2;
    if (o < nS) {
      // lower-triangle index o -> (ii, cc), cc <= ii (o < 1176: the float root is exact enough)
      int ii = (int)((sqrtf(8.0f * (float)o + 1.0f) - 1.0f) * 0.5f);
      while ((ii + 1) * (ii + 2) / 2 <= o) ii++;
      while (ii * (ii + 1) / 2 > o) ii--;
      const int cc = o - ii * (ii + 1) / 2;
      const int i = c0 + kPbB + ii, c = c0 + kPbB + cc;
      T acc0 = S(i, c), acc1 = AR::zero();
#pragma unroll
      for (int j = 0; j < kPbB; j += 2) {
        acc0 = AR::fnma_lazy(acc0, Tm[ii * kPbB + j], S(c, c0 + j));
        acc1 = AR::fnma_lazy(acc1, Tm[ii * kPbB + j + 1], S(c, c0 + j + 1));
      }
      S(i, c) = AR::add(acc0, acc1);
    } else {
      const int oo = o - nS;
      const int ii = oo / cw, c = oo % cw;
      const int i = c0 + kPbB + ii;
      T acc0 = Y(i, c), acc1 = AR::zero();
      const int j0 = (c > c0) ? c - c0 : 0;          // Y[c0 + j][c] = 0 for c > c0 + j
      for (int j = j0; j < kPbB; j += 2) {
        const T y0 = (c0 + j == c) ? AR::one() : Y(c0 + j, c);
        acc0 = AR::fnma_lazy(acc0, Tm[ii * kPbB + j], y0);
        if (j + 1 < kPbB) acc1 = AR::fnma_lazy(acc1, Tm[ii * kPbB + j + 1], Y(c0 + j + 1, c));
      }
      Y(i, c) = AR::add(acc0, acc1);
    }
  };
  constexpr int kDiagOut = kPbB * (kPbB + 1) / 2;   // the next diagonal block's outputs
  int pend = -1;                                    // sub-panel whose trailing update is unfinished

  for (int p = 0; p < NB / kPbB; p++) {
    const int c0 = p * kPbB;
    // ---- the rest of the previous sub-panel's trailing update (everything but this sub-panel's
    //      diagonal block, which the sweep below needs and which was updated first), by the 768
    //      threads the sweep leaves idle: it touches neither the block nor the sweep's buffers
    if (t >= kPbB * kPbB && pend >= 0) {
      const int nr = NB - pend - kPbB;
      const int tot = nr * (nr + 1) / 2 + nr * (pend + kPbB);
      for (int o = kDiagOut + (t - kPbB * kPbB); o < tot; o += kPbThreads - kPbB * kPbB) trailing(pend, o);
    }
    // ---- (a) the 16 x 16 diagonal sub-block, by the first 256 threads (8 warps, one named
    //      barrier per column): thread (r, cl) holds element (c0 + r, c0 + cl), S until column
    //      cl is published, then Y.  One element per thread keeps each step's dependent chain
    //      (pivot reciprocal, multiplier, one fused update) short in every warp.
    if (t < kPbB * kPbB) {
      const int r = t / kPbB, cl = t % kPbB, i = c0 + r;
      T X = (cl <= r) ? S(i, c0 + cl) : AR::zero();
      bool ok = true;
      for (int jj = 0; jj < kPbB; jj++) {
        T* cb = colbuf + (jj & 1) * kPbB;
        T* rb = rowbuf + (jj & 1) * kPbB;
        if (cl == jj && r >= jj) {        // the owner of column jj publishes it
          cb[r] = X;
          S(i, c0 + jj) = X;
          X = AR::zero();                 // from here on the register accumulates Y[i][c0 + jj]
        }
        if (r == jj && cl < jj) rb[cl] = X;
        asm volatile("bar.sync 1, %0;" ::"r"(kPbB * kPbB) : "memory");
        const T d = cb[jj];
        if (!AR::positive(d)) {   // every thread reads the same pivot: the exit is uniform
          ok = false;
          break;
        }
        const T rcpd = AR::rcp(d);
        if (t == 0) rd[c0 + jj] = rcpd;
        if (r > jj && cl <= r) {
          const T a = AR::mul(cb[r], rcpd);
          const T v = (cl > jj) ? cb[cl] : (cl == jj ? AR::one() : rb[cl]);
          X = AR::fnma(X, a, v);
        }
      }
      if (!ok) {
        if (t == 0) *bad = 1;
      } else if (cl < r) {
        Y(i, c0 + cl) = X;
      }
    }
    __syncthreads();
    if (*bad) {
      if (t == 0) atomicExch(flag, 1);
      return;
    }
    // ---- (b) into registers: S21 = B21 Y_pp^T (rows below, sub-panel columns) and the
    //      sub-panel rows' Y on the earlier columns, Y_pp Y_old
    const int nb_rows = NB - c0 - kPbB;                // rows below the sub-panel
    const int n21 = nb_rows * kPbB, nya = kPbB * c0;
    constexpr int kRegs = (3 * kPbB * kPbB + kPbThreads - 1) / kPbThreads;   // outputs per thread, at most
    T vb[kRegs];
#pragma unroll
    for (int q = 0; q < kRegs; q++) {
      const int o = t + q * kPbThreads;
      vb[q] = AR::zero();
      if (o < n21) {
        const int i = c0 + kPbB + o / kPbB, j = o % kPbB;
        T acc0 = AR::zero(), acc1 = AR::zero();
        for (int c = 0; c <= j; c += 2) {   // Y_pp[j][c] (unit diagonal)
          const T y0 = (c == j) ? AR::one() : Y(c0 + j, c0 + c);
          acc0 = AR::fnma_lazy(acc0, S(i, c0 + c), y0);
          if (c + 1 <= j) {
            const T y1 = (c + 1 == j) ? AR::one() : Y(c0 + j, c0 + c + 1);
            acc1 = AR::fnma_lazy(acc1, S(i, c0 + c + 1), y1);
          }
        }
        const T acc = AR::add(acc0, acc1);
        vb[q] = {-acc.h, -acc.l};
      } else if (o < n21 + nya) {
        const int oo = o - n21;
        const int i = c0 + oo / c0, c = oo % c0;
        T acc0 = AR::zero(), acc1 = AR::zero();
        for (int j = c0; j <= i; j += 2) {  // sum_j Y_pp[i][j] Y_old[j][c]
          const T y0 = (j == i) ? AR::one() : Y(i, j);
          acc0 = AR::fnma_lazy(acc0, y0, Y(j, c));
          if (j + 1 <= i) {
            const T y1 = (j + 1 == i) ? AR::one() : Y(i, j + 1);
            acc1 = AR::fnma_lazy(acc1, y1, Y(j + 1, c));
          }
        }
        const T acc = AR::add(acc0, acc1);
        vb[q] = {-acc.h, -acc.l};
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kRegs; q++) {
      const int o = t + q * kPbThreads;
      if (o < n21) {
        const int ii = o / kPbB, j = o % kPbB;
        S(c0 + kPbB + ii, c0 + j) = vb[q];
        Tm[ii * kPbB + j] = AR::mul(vb[q], rd[c0 + j]);
      } else if (o < n21 + nya) {
        const int oo = o - n21;
        Y(c0 + oo / c0, oo % c0) = vb[q];
      }
    }
    __syncthreads();
    if (nb_rows == 0) break;
    // ---- (c) trailing rank-16 update of the rows below: S22 -= T21 S21^T (lower), and
    //      Y_below[:, < c0 + 16] -= T21 Y_p.  Only the next sub-panel's diagonal block now; the
    //      rest runs beside the next sweep (above), before the next phase (b) reads it.
    for (int o = t; o < kDiagOut; o += kPbThreads) trailing(c0, o);
    pend = c0;
    __syncthreads();
  }
  // ---- outputs: L' = S diag(1/sqrt(d)), L'^{-1} = diag(1/sqrt(d)) Y, unscaled by D
  if (t < NB) rsd[t] = AR::rsqrt(S(t, t));
  __syncthreads();
  float2* Lf2 = LinvDF + (k0 / NB) * NB * NB;
  float2* Ld2 = LDF + (k0 / NB) * NB * NB;
  for (int idx = t; idx < NB * NB; idx += kPbThreads) {
    const int i = idx / NB, c = idx % NB;
    const bool in = i < kb && c <= i;
    T v = AR::zero(), l = AR::zero();
    if (in) {
      v = (c == i) ? rsd[i] : AR::mul(Y(i, c), rsd[i]);   // L'^{-1}[i][c] = Y[i][c] / sqrt(d_i)
      l = AR::mul(S(i, c), rsd[c]);                       // L'[i][c] = S[i][c] / sqrt(d_c)
    }
    Lf2[idx] = make_float2(v.h, v.l);
    Ld2[idx] = make_float2(l.h, l.l);
  }
  if (t < NB) scOut[(k0 / NB) * NB + t] = sc[t];
  if (fw) {
    // forward substitution, block k: y_k = L'^{-1} (D w_k); 16 threads per row, combined by shuffles
    constexpr int kTpr = kPbThreads / NB;
    const int i = t / kTpr, g = t % kTpr;
    T acc = AR::zero();
    if (i < kb) {
      for (int c = g; c <= i; c += kTpr) {
        const T v = (c == i) ? rsd[i] : AR::mul(Y(i, c), rsd[i]);
        acc = AR::add(acc, AR::mul(v, AR::load_scaled(fw[k0 + c], nullptr, -sc[c])));
      }
    }
#pragma unroll
    for (int o = 1; o < kTpr; o <<= 1) {
      const T other = {__shfl_xor_sync(0xffffffffu, acc.h, o), __shfl_xor_sync(0xffffffffu, acc.l, o)};
      acc = AR::add(acc, other);
    }
    if (g == 0 && i < kb) {
      fy[k0 + i] = AR::store_scaled(acc, 0);
      fyDF[i] = make_float2(acc.h, acc.l);
    }
  }
}

// The FP64 copies of every diagonal block's factor, from the double-float results of
// potrf_blk_kernel: L = D^-1 L' into A's diagonal block (lower, rows < kb) and
// Linv = L'^{-1} D (the full 64 x 64, zero above the diagonal and on the padding).  One CTA per
// block.
__global__ void __launch_bounds__(256) diag_to_fp64_kernel(double* A, int64_t lda, int64_t n, const float2* LDF,
                                                            const float2* LinvDF, const int* sc, double* Linv,
                                                            const int* flag) {
  if (*flag) return;
  const int64_t k = blockIdx.x, k0 = k * NB;
  const int kb = (int)((n - k0) < NB ? (n - k0) : NB);
  const float2* Ld = LDF + k * NB * NB;
  const float2* Lv = LinvDF + k * NB * NB;
  const int* s = sc + k * NB;
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    const int i = idx / NB, c = idx % NB;
    const bool in = i < kb && c <= i;
    const float2 v = Lv[idx];
    Linv[k * NB * NB + idx] = in ? ArithDF::store_scaled({v.x, v.y}, -s[c]) : 0.0;
    if (in) {
      const float2 l = Ld[idx];
      A[(k0 + i) * lda + k0 + c] = ArithDF::store_scaled({l.x, l.y}, s[i]);
    }
  }
}

// Panel solve L21 = A21 Linv_k^T in FP64 on the CUDA cores (the FP64 path), in
// place, for the rows [k1, n) of the panel columns [k0, k0 + kb).  32 rows per
// CTA, 128 threads, 4 x 4 outputs per thread (rows ty + 8a, columns tx + 16b);
// Linv_k is lower triangular, so the K loop runs in four 16-wide segments and
// segment s only feeds the columns b >= s.
constexpr int kPanelRows = 32;
constexpr size_t kPanelSmem = (size_t)(kPanelRows + NB) * (NB + 1) * 8;

__global__ void __launch_bounds__(128) panel_solve_kernel(double* A, int64_t lda, int64_t k0, int kb, int64_t k1,
                                                          int64_t n, const double* __restrict__ Lk, const int* flag) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double (*As)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(smraw);
  double (*Lt)[NB + 1] = As + kPanelRows;   // Lt[q][j] = Linv_k[j][q]
  if (*flag) return;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int64_t rb = k1 + (int64_t)blockIdx.x * kPanelRows;   // first row of this CTA
  for (int idx = t; idx < NB * NB; idx += blockDim.x) {
    const int j = idx / NB, q = idx % NB;
    Lt[q][j] = (j < kb && q < kb) ? Lk[j * NB + q] : 0.0;
  }
  for (int idx = t; idx < kPanelRows * NB; idx += blockDim.x) {
    const int rr = idx / NB, q = idx % NB;
    const int64_t r = rb + rr;
    As[rr][q] = (r < n && q < kb) ? A[r * lda + k0 + q] : 0.0;
  }
  __syncthreads();
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
#pragma unroll
  for (int seg = 0; seg < 4; seg++) {
#pragma unroll 4
    for (int tt = 0; tt < 16; tt++) {
      const int q = 16 * seg + tt;
      double av[4], lv[4];
#pragma unroll
      for (int a = 0; a < 4; a++) av[a] = As[ty + 8 * a][q];
#pragma unroll
      for (int b = seg; b < 4; b++) lv[b] = Lt[q][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = seg; b < 4; b++) acc[a][b] = fma(av[a], lv[b], acc[a][b]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int64_t r = rb + ty + 8 * a;
    if (r >= n) continue;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int j = tx + 16 * b;
      if (j >= kb) continue;
      A[r * lda + k0 + j] = acc[a][b];
    }
  }
}

// The split path's panel solve in double-float arithmetic on the FP32 pipe
// (about 48 significant bits, the precision of U and of the split GEMM):
// L21 = (A21 - U21) D L'^{-T}, with L'^{-1} (LkDF) and the power-of-two scales
// D = diag(2^-sc) from the diagonal factor.  16 rows per CTA (enough CTAs for about three per
// SM, whose warps hide each other's latency), 256 threads, 1 x 4 outputs per thread (row ty,
// columns tx + 16b), the same K segments as the FP64 kernel;
// each product is the exact FP32 product of the high parts plus the cross
// terms, its high part added exactly (TwoSum) and the low parts accumulated
// in FP32, renormalised at the end.  Writes L21 in FP64 and its S BF16 slices
// into the strip operand (row r at r - row_base, columns kofs + j), with each
// row's own exponent over this panel's 64 columns in eout[r - row_base] (the
// strip operand keeps one exponent array per panel).
constexpr int kPanelDFRowsCTA = 16;                       // rows per CTA: about three CTAs per SM
constexpr size_t kPanelDFSmem = (size_t)(kPanelDFRowsCTA + NB) * (NB + 1) * sizeof(float2);
constexpr int kPanelDFThreads = 256;                       // 16 x 16: 1 row x 4 columns per thread
constexpr int kPanelDFRowStride = kPanelDFThreads / 16;    // rows ty + 16 a
constexpr int kPanelDFRows = kPanelDFRowsCTA / kPanelDFRowStride;

template <int S>
__global__ void __launch_bounds__(kPanelDFThreads) panel_df_kernel(double* A, int64_t lda, int64_t k0, int kb, int64_t k1,
                                                       int64_t n, const float2* __restrict__ U, int64_t ldu,
                                                       const float2* __restrict__ LkDF, const int* __restrict__ sck,
                                                       __nv_bfloat16* slices, int* eout, int64_t row_base,
                                                       int64_t npad, int64_t kpad, int kofs,
                                                       const float2* __restrict__ fyDF, double* fw, const int* flag) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2 (*As)[NB + 1] = reinterpret_cast<float2 (*)[NB + 1]>(smraw);
  float2 (*Lt)[NB + 1] = As + kPanelDFRowsCTA;   // Lt[q][j] = L'^{-1}[j][q]
  __shared__ float colscale[NB];   // 2^-sc[q]; 0 marks a scale outside FP32's range
  if (*flag) return;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int64_t rb = k1 + (int64_t)blockIdx.x * kPanelDFRowsCTA;
  // every global load of the CTA is issued before any is consumed (the panel is latency-bound):
  // L'^{-1} (16 values per thread) and the panel rows A, U (8 values per thread)
  constexpr int kLtPer = NB * NB / kPanelDFThreads, kAsPer = kPanelDFRowsCTA * NB / kPanelDFThreads;
  float2 ltv[kLtPer];
  double av[kAsPer];
  float2 uv[kAsPer];
#pragma unroll
  for (int m = 0; m < kLtPer; m++) {
    const int idx = t + m * kPanelDFThreads, j = idx / NB, q = idx % NB;
    ltv[m] = (j < kb && q < kb) ? LkDF[j * NB + q] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int m = 0; m < kAsPer; m++) {
    const int idx = t + m * kPanelDFThreads, rr = idx / NB, q = idx % NB;
    const int64_t r = rb + rr;
    const bool in = r < n && q < kb;
    av[m] = in ? A[r * lda + k0 + q] : 0.0;
    uv[m] = (in && U) ? U[r * ldu + k0 + q] : make_float2(0.f, 0.f);
  }
  if (t < NB) colscale[t] = (t < kb && sck[t] >= -120 && sck[t] <= 120) ? ldexpf(1.0f, -sck[t]) : 0.0f;
#pragma unroll
  for (int m = 0; m < kLtPer; m++) {
    const int idx = t + m * kPanelDFThreads;
    Lt[idx % NB][idx / NB] = ltv[m];
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < kAsPer; m++) {
    const int idx = t + m * kPanelDFThreads, rr = idx / NB, q = idx % NB;
    const int64_t r = rb + rr;
    float h = 0.f, l = 0.f;
    if (r < n && q < kb && colscale[q] == 0.0f) {   // extreme scale: subtract and scale in FP64
      double a = av[m];
      if (U) {
        const float2 u = uv[m];
        a -= (double)u.x + (double)u.y;
      }
      a *= p2(-sck[q]);
      h = __double2float_rn(a);
      l = __double2float_rn(a - (double)h);
    } else if (r < n && q < kb) {
      const double a = av[m];
      h = __double2float_rn(a);
      l = __double2float_rn(a - (double)h);
      if (U) {   // (h, l) -= (u.x, u.y): TwoSum of the high parts, low parts added
        const float2 u = uv[m];
        const float s1 = __fsub_rn(h, u.x);
        const float bb = __fsub_rn(s1, h);
        const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s1, bb)), __fsub_rn(-u.x, bb));
        const float tl = __fadd_rn(err, __fsub_rn(l, u.y));
        h = __fadd_rn(s1, tl);
        l = __fsub_rn(tl, __fsub_rn(h, s1));
      }
      const float sc = colscale[q];   // exact power of two
      h = __fmul_rn(h, sc);
      l = __fmul_rn(l, sc);
    }
    As[rr][q] = make_float2(h, l);
  }
  __syncthreads();
  float ah[kPanelDFRows][4], al[kPanelDFRows][4];
#pragma unroll
  for (int a = 0; a < kPanelDFRows; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) ah[a][b] = al[a][b] = 0.f;
#pragma unroll
  for (int seg = 0; seg < 4; seg++) {
#pragma unroll 2
    for (int tt = 0; tt < 16; tt++) {
      const int q = 16 * seg + tt;
      float2 av[kPanelDFRows], lv[4];
#pragma unroll
      for (int a = 0; a < kPanelDFRows; a++) av[a] = As[ty + kPanelDFRowStride * a][q];
#pragma unroll
      for (int b = seg; b < 4; b++) lv[b] = Lt[q][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < kPanelDFRows; a++)
#pragma unroll
        for (int b = seg; b < 4; b++) {
          const float p = __fmul_rn(av[a].x, lv[b].x);
          float pe = __fmaf_rn(av[a].x, lv[b].x, -p);
          pe = __fmaf_rn(av[a].x, lv[b].y, __fmaf_rn(av[a].y, lv[b].x, pe));
          const float s1 = __fadd_rn(ah[a][b], p);
          const float bb = __fsub_rn(s1, ah[a][b]);
          const float err = __fadd_rn(__fsub_rn(ah[a][b], __fsub_rn(s1, bb)), __fsub_rn(p, bb));
          ah[a][b] = s1;
          al[a][b] = __fadd_rn(al[a][b], __fadd_rn(pe, err));
        }
    }
  }
#pragma unroll
  for (int a = 0; a < kPanelDFRows; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) {   // renormalise (Fast2Sum)
      const float hi = __fadd_rn(ah[a][b], al[a][b]);
      al[a][b] = __fsub_rn(al[a][b], __fsub_rn(hi, ah[a][b]));
      ah[a][b] = hi;
    }
  if (fw) {
    // forward substitution: w[r] -= L21[r][:] y_k, the 16 lanes of a row (a half warp) combining
#pragma unroll
    for (int a = 0; a < kPanelDFRows; a++) {
      DF acc = {0.f, 0.f};
#pragma unroll
      for (int b = 0; b < 4; b++) {
        const int j = tx + 16 * b;
        if (j < kb) {
          const float2 yv = fyDF[j];
          acc = ArithDF::add(acc, ArithDF::mul({ah[a][b], al[a][b]}, {yv.x, yv.y}));
        }
      }
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) {
        const DF other = {__shfl_xor_sync(0xffffffffu, acc.h, o), __shfl_xor_sync(0xffffffffu, acc.l, o)};
        acc = ArithDF::add(acc, other);
      }
      const int64_t r = rb + ty + kPanelDFRowStride * a;
      if (tx == 0 && r < n) fw[r] = (fw[r] - (double)acc.h) - (double)acc.l;
    }
  }
#pragma unroll
  for (int a = 0; a < kPanelDFRows; a++) {
    const int64_t r = rb + ty + kPanelDFRowStride * a;
    // row maximum over the 16 lanes holding this row (a half warp); |hi| suffices: with
    // 2^e > max |hi| the leading digit stays <= 2^8, exact in BF16
    float m = 0.f;
#pragma unroll
    for (int b = 0; b < 4; b++)
      if (tx + 16 * b < kb) m = fmaxf(m, fabsf(ah[a][b]));
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    int e = 0;
    if (m > 0.f && isfinite(m)) frexpf(m, &e);
    if (r >= n) continue;
    if (tx == 0) eout[r - row_base] = e;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int j = tx + 16 * b;
      if (j >= kb) continue;
      const double x = (double)ah[a][b] + (double)al[a][b];
      A[r * lda + k0 + j] = x;
      oz_digits<S>(x, e, slices + (r - row_base) * kpad + kofs + j, npad * kpad);
    }
  }
}

// Blocked triangular solves with the stored diagonal inverses.  One launch per
// block: every CTA forms z = Linv_k w_k (or Linv_k^T w_k) itself from the 64
// values of w it reads (2080 FMAs, cheaper than a second launch), CTA 0 stores
// z, and all CTAs apply it to their rows of the remaining vector.  w is the
// work vector; z goes to a separate output, so no CTA overwrites values
// another CTA of the same launch still reads.
constexpr int kSolveThreads = 256;

__device__ __forceinline__ void block_tri(const double* __restrict__ Lk, const double* __restrict__ wk, int kb,
                                          int trans, double (*Ls)[NB + 1], double* ws, double* zs) {
  const int t = threadIdx.x;
  // stage Linv_k in shared memory: 16 independent loads per thread, all in flight together
#pragma unroll
  for (int m = 0; m < NB * NB / kSolveThreads; m++) {
    const int idx = t + m * kSolveThreads;
    Ls[idx / NB][idx % NB] = Lk[idx];
  }
  if (t < NB) ws[t] = (t < kb) ? wk[t] : 0.0;
  __syncthreads();
  const int i = t >> 2, part = t & 3;   // 4 threads per output row
  double acc = 0.0;
  if (i < kb) {
    if (!trans) {
      for (int q = part; q <= i; q += 4) acc = fma(Ls[i][q], ws[q], acc);
    } else {
      for (int q = i + part; q < kb; q += 4) acc = fma(Ls[q][i], ws[q], acc);
    }
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  if (part == 0) zs[i] = acc;
  __syncthreads();
}

// forward block k: y_k = Linv_k w_k; w[r] -= sum_t L[r][k0 + t] y_k[t] for rows r >= k1 (one warp per row)
__global__ void __launch_bounds__(kSolveThreads) fwd_step_kernel(const double* __restrict__ L, int64_t lda,
                                                                 const double* __restrict__ Lk, double* w,
                                                                 double* y, int64_t k0, int kb, int64_t n) {
  __shared__ double Ls[NB][NB + 1], ws[NB], zs[NB];
  block_tri(Lk, w + k0, kb, 0, Ls, ws, zs);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (blockIdx.x == 0 && t < kb) y[k0 + t] = zs[t];
  const int64_t k1 = k0 + kb;
  for (int64_t row = k1 + (int64_t)blockIdx.x * 8 + warp; row < n; row += (int64_t)gridDim.x * 8) {
    double acc = 0.0;
    for (int q = lane; q < kb; q += 32) acc = fma(L[row * lda + k0 + q], zs[q], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) w[row] -= acc;
  }
}

// backward block k: x_k = Linv_k^T w_k; w[j] -= sum_t L[k0 + t][j] x_k[t] for j < k0.
// 64 values of j per CTA, 4 threads per j (16 t each, coalesced over j), partial
// sums combined in shared memory: FP64 work is spread over many SMs.
__global__ void __launch_bounds__(kSolveThreads) bwd_step_kernel(const double* __restrict__ L, int64_t lda,
                                                                 const double* __restrict__ Lk, double* w,
                                                                 double* x, int64_t k0, int kb) {
  __shared__ double Ls[NB][NB + 1], ws[NB], zs[NB];
  __shared__ double part[4][NB];
  block_tri(Lk, w + k0, kb, 1, Ls, ws, zs);
  const int t = threadIdx.x;
  if (blockIdx.x == 0 && t < kb) x[k0 + t] = zs[t];
  const int jj = t & (NB - 1), qp = t >> 6;
  const int64_t j = (int64_t)blockIdx.x * NB + jj;
  double acc0 = 0.0, acc1 = 0.0;
  if (j < k0) {
#pragma unroll
    for (int u = 0; u < 16; u += 2) {
      const int q0 = qp * 16 + u, q1 = q0 + 1;
      if (q0 < kb) acc0 = fma(L[(k0 + q0) * lda + j], zs[q0], acc0);
      if (q1 < kb) acc1 = fma(L[(k0 + q1) * lda + j], zs[q1], acc1);
    }
  }
  part[qp][jj] = acc0 + acc1;
  __syncthreads();
  if (t < NB && j < k0) w[j] -= (part[0][jj] + part[1][jj]) + (part[2][jj] + part[3][jj]);
}

}  // namespace

namespace {

template <class AR>
cudaError_t launch_potrf(double* A, int64_t lda, int64_t k0, int kb, const float2* U, int64_t ldu, double* Linv,
                         float2* LinvDF, int* scOut, const double* fw, double* fy, float2* fyDF, int* flag,
                         cudaStream_t st) {
  static_assert(kPotrfSmem <= 48 * 1024, "the diagonal factor's shared memory needs no opt-in");
  potrf_inv_kernel<AR, kPotrfTPR><<<1, NB * kPotrfTPR, kPotrfSmem, st>>>(A, lda, k0, kb, U, ldu, Linv, LinvDF, scOut,
                                                                          fw, fy, fyDF, flag);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_potrf_blk(const double* A, int64_t lda, int64_t k0, int kb, const float2* U, int64_t ldu,
                             float2* LDF, float2* LinvDF, int* scOut, const double* fw, double* fy, float2* fyDF,
                             int* flag, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(potrf_blk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPbSmem);
  if (e != cudaSuccess) return e;
  potrf_blk_kernel<<<1, kPbThreads, kPbSmem, st>>>(A, lda, k0, kb, U, ldu, LDF, LinvDF, scOut, fw, fy, fyDF, flag);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_panel(double* A, int64_t lda, int64_t k0, int kb, int64_t k1, int64_t n, const double* Lk,
                         const int* flag, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(panel_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kPanelSmem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (n - k1 + kPanelDFRowsCTA - 1) / kPanelDFRowsCTA;
  if (blocks <= 0) return cudaSuccess;
  panel_solve_kernel<<<(unsigned)blocks, 128, kPanelSmem, st>>>(A, lda, k0, kb, k1, n, Lk, flag);
  count_launch();
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_panel_df(double* A, int64_t lda, int64_t k0, int kb, int64_t k1, int64_t n, const float2* U,
                            int64_t ldu, const float2* LkDF, const int* sck, const OzOperand& op, int* eout,
                            int64_t row_base, int kofs, const float2* fyDF, double* fw, const int* flag,
                            cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(panel_df_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kPanelDFSmem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (n - k1 + kPanelDFRowsCTA - 1) / kPanelDFRowsCTA;
  if (blocks <= 0) return cudaSuccess;
  panel_df_kernel<S><<<(unsigned)blocks, kPanelDFThreads, kPanelDFSmem, st>>>(A, lda, k0, kb, k1, n, U, ldu, LkDF, sck,
                                                                  static_cast<__nv_bfloat16*>(op.slices), eout,
                                                                  row_base, op.npad, op.kpad, kofs, fyDF, fw,
                                                                  flag);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_panel_split(int S, double* A, int64_t lda, int64_t k0, int kb, int64_t k1, int64_t n,
                               const float2* U, int64_t ldu, const float2* LkDF, const int* sck, const OzOperand& op,
                               int* eout, int64_t row_base, int kofs, const float2* fyDF, double* fw,
                               const int* flag, cudaStream_t st) {
  switch (S) {
#define GN_PANEL_CASE(s)                                                                                   \
  case s:                                                                                                  \
    return launch_panel_df<s>(A, lda, k0, kb, k1, n, U, ldu, LkDF, sck, op, eout, row_base, kofs, fyDF, fw, \
                              flag, st);
    GN_PANEL_CASE(1)
    GN_PANEL_CASE(2)
    GN_PANEL_CASE(3)
    GN_PANEL_CASE(4)
    GN_PANEL_CASE(5)
    GN_PANEL_CASE(6)
#undef GN_PANEL_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t cholesky_factor(double* A, int64_t n, int64_t lda, double* Linv, int* flag, cudaStream_t st) {
  cudaError_t err = cudaSuccess;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int kb = (int)((n - k0) < NB ? (n - k0) : NB);
    if ((err = launch_potrf<Arith64>(A, lda, k0, kb, nullptr, 0, Linv, nullptr, nullptr, nullptr, nullptr, nullptr,
                                     flag, st)) != cudaSuccess)
      return err;
    const int64_t k1 = k0 + kb;
    if (k1 >= n) break;
    const double* Lk = Linv + (k0 / NB) * NB * NB;
    // panel: A21 <- A21 Linv_k^T
    if ((err = launch_panel(A, lda, k0, kb, k1, n, Lk, flag, st)) != cudaSuccess) return err;
    // trailing: A22 -= L21 L21^T (lower)
    err = dgemm(n - k1, n - k1, kb, -1.0, A + k1 * lda + k0, lda, true, A + k1 * lda + k0, lda, true, 1.0,
                A + k1 * lda + k1, lda, true, nullptr, st);
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

// Same blocked factorisation with the trailing updates on the tensor cores
// (split GEMM, S slices).  U, the double-FP32 sum of all updates so far
// (n x n float2), is accumulated on the FP32 pipe by the split GEMM's
// epilogue; the diagonal factor and the panel solve subtract it from the 64
// columns they read, so the FP64 work of the updates drops from O(n^3/64) to
// O(n^2).
//
// Two-level blocking: the 64-wide panels are grouped in strips of kStrip = 256
// columns.  Each panel writes its slices into the strip's operand with its own
// row exponents (one exponent array per panel: the split GEMM applies them per
// 64-column chunk), so the bulk update of the trailing matrix runs once per
// strip (one split GEMM with K = 256, a quarter of the passes over U) at the
// precision of per-panel updates.  Inside the strip, each panel's own 64
// columns first get the updates of the strip's earlier panels (a 64-column
// split GEMM over the chunks already written).
//
// Look-ahead: the bulk update of strip t is split into the next strip's 256
// columns, done at once on the critical stream, and the rest, deferred to a
// low-priority stream where it overlaps strip t + 1's chain (which touches only
// its own columns).  Strip operands alternate between two buffers.
//
// The diagonal blocks and the panels are computed in double-float arithmetic
// (about 48 significant bits, the precision U and the split GEMM carry).
// With a right-hand side b, the forward substitution L y = b rides along: the
// diagonal factor forms y_k = Linv_k w_k and the panel kernel applies it to
// the rows below (w: n doubles of work space, y: n doubles out).
// *rc_out receives a GN_ERR_* code on failure.
constexpr int64_t kStrip = kCholStrip;

// Split workspace of cholesky_factor_split: U (n x n double-FP32), two strip operands
// (slices and four exponent arrays each), the double-float diagonal factors and inverses, their
// scales and the double-float forward-solve block.
size_t chol_split_ws_bytes(int64_t n, int S) {
  auto rup = [](int64_t v, int64_t m) { return (v + m - 1) / m * m; };
  const int64_t npad0 = rup(n, 128);
  const size_t ub = rup((int64_t)n * n * sizeof(float2), 256);
  const size_t sb = rup((int64_t)S * npad0 * kStrip * 2, 256);
  const int64_t estride = npad0 + 1024;
  const size_t eb = rup(4 * estride * sizeof(int), 256);
  const int64_t nblk = (n + NB - 1) / NB;
  const size_t lb = rup(nblk * NB * NB * sizeof(float2), 256);
  const size_t cb = rup(nblk * NB * sizeof(int), 256);
  const size_t yb = rup(NB * sizeof(float2), 256);
  return ub + 2 * (sb + eb) + 2 * lb + cb + yb + 256;
}

// The look-ahead's streams: the critical path at the highest priority, the deferred bulk
// updates in the middle, and the pipelined step's Gram chunks at the lowest (numerically
// greater is lower; with only two levels the last two share one).
cudaError_t ensure_chol_streams(gn_handle* h) {
  if (h->st_hi) return cudaSuccess;
  int least = 0, greatest = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  const int middle = greatest + (least - greatest + 1) / 2;
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->st_hi, cudaStreamNonBlocking, greatest);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->st_lo, cudaStreamNonBlocking, middle);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->st_g, cudaStreamNonBlocking, least);
  return e;
}

int ensure_chol_ws(gn_handle* h, size_t need) {
  if (h->chol_ws_bytes >= need) return GN_OK;
  if (h->capturing) {   // prepare_for_capture sized it; growing now would allocate inside a capture
    set_detail(__FILE__, __LINE__, "factorisation workspace would grow during a graph capture");
    return GN_ERR_UNSUPPORTED;
  }
  if (h->chol_ws) cudaFree(h->chol_ws);   // synchronises: no kernel still reads it
  h->chol_ws = nullptr;
  h->chol_ws_bytes = 0;
  if (GN_NOTE(cudaMalloc(&h->chol_ws, need)) != cudaSuccess) return GN_ERR_OOM;
  h->chol_ws_bytes = need;
  return GN_OK;
}

cudaError_t cholesky_factor_split(gn_handle* h, double* A, int64_t n, int64_t lda, double* Linv, int* flag, int S,
                                  const double* b, double* y, double* w, int* rc_out, const cudaEvent_t* gate) {
  cudaStream_t st = h->st;
  *rc_out = GN_OK;
  auto rup = [](int64_t v, int64_t m) { return (v + m - 1) / m * m; };
  const int64_t npad0 = rup(n, 128);
  const size_t ub = rup((int64_t)n * n * sizeof(float2), 256);
  const size_t sb = rup((int64_t)S * npad0 * kStrip * 2, 256);      // one strip operand's slices
  const int64_t estride = npad0 + 1024;                             // exponent rows per panel chunk, padded
  const size_t eb = rup(4 * estride * sizeof(int), 256);            // one strip operand's 4 exponent arrays
  const int64_t nblk = (n + NB - 1) / NB;
  const size_t lb = rup(nblk * NB * NB * sizeof(float2), 256);
  const size_t cb = rup(nblk * NB * sizeof(int), 256);
  int rc = ensure_chol_ws(h, chol_split_ws_bytes(n, S));
  if (rc) {
    *rc_out = rc;
    return cudaErrorMemoryAllocation;
  }
  unsigned char* base = static_cast<unsigned char*>(h->chol_ws);
  float2* U = reinterpret_cast<float2*>(base);
  unsigned char* strip_base = base + ub;   // two strip operands of sb + eb bytes
  float2* LinvDF = reinterpret_cast<float2*>(base + ub + 2 * (sb + eb));
  int* scales = reinterpret_cast<int*>(base + ub + 2 * (sb + eb) + lb);
  float2* yDF = reinterpret_cast<float2*>(base + ub + 2 * (sb + eb) + lb + cb);
  float2* LDF = reinterpret_cast<float2*>(base + ub + 2 * (sb + eb) + lb + cb + rup(NB * sizeof(float2), 256));
  {
    const cudaError_t e = ensure_chol_streams(h);
    if (e != cudaSuccess) return e;
  }
  cudaStream_t sh = h->st_hi, sl = h->st_lo;
  const int64_t nstrip = (n + kStrip - 1) / kStrip;
  std::vector<cudaEvent_t> evs(2 * nstrip + 3, nullptr);
  cudaError_t err = cudaSuccess;
  for (auto& e : evs)
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  struct Guard {   // events may be destroyed while work on them is pending
    std::vector<cudaEvent_t>& v;
    ~Guard() {
      for (auto e : v)
        if (e) cudaEventDestroy(e);
    }
  } guard{evs};
  if (err != cudaSuccess) return err;
  cudaEvent_t* evA = evs.data();            // [t]: strip t's next-columns update done
  cudaEvent_t* evB = evs.data() + nstrip;   // [t]: strip t's deferred bulk update done
  cudaEvent_t e0 = evs[2 * nstrip], e_hi = evs[2 * nstrip + 1], e_lo = evs[2 * nstrip + 2];
  std::vector<char> launchedB(nstrip, 0);
  auto fail = [&](int code) {
    *rc_out = code;
    return cudaErrorUnknown;
  };
  if ((err = cudaEventRecord(e0, st)) != cudaSuccess) return err;
  if ((err = cudaStreamWaitEvent(sh, e0, 0)) != cudaSuccess) return err;
  if ((err = cudaStreamWaitEvent(sl, e0, 0)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(U, 0, (size_t)n * n * sizeof(float2), sh)) != cudaSuccess) return err;
  if (b && (err = cudaMemcpyAsync(w, b, n * sizeof(double), cudaMemcpyDeviceToDevice, sh)) != cudaSuccess) return err;
  cudaEvent_t waited = nullptr;
  for (int64_t t = 0; t < nstrip; t++) {
    const int64_t s0 = t * kStrip;
    const int64_t s1 = (s0 + kStrip < n) ? s0 + kStrip : n;
    // the strip's columns of A may still be in production (pipelined step)
    if (gate && gate[t] && gate[t] != waited) {
      if ((err = cudaStreamWaitEvent(sh, gate[t], 0)) != cudaSuccess) return err;
      waited = gate[t];
    }
    // strip operand t % 2 (rows relative to s0); its previous user, strip t - 2's deferred
    // update, finished before strip t - 1's next-columns update (the wait below)
    unsigned char* sbase = strip_base + (t & 1) * (sb + eb);
    OzOperand strip;
    strip.slices = sbase;
    strip.e = reinterpret_cast<int*>(sbase + sb);
    strip.npad = rup(n - s0, 128);
    strip.kpad = kStrip;
    strip.echunk = NB;
    strip.estride = estride;
    // the strip's chain: in-strip updates, diagonal factors, panels
    for (int64_t k0 = s0; k0 < s1; k0 += NB) {
      const int kb = (int)((n - k0) < NB ? (n - k0) : NB);
      const int kofs = (int)(k0 - s0);
      if (kofs > 0) {
        // U[k0:, k0:k0+kb] += L[k0:, s0:k0] L[k0:k0+kb, s0:k0]^T (64 columns: 128 x 64 tiles)
        OzOperand v = oz_operand_rows(strip, S, k0 - s0);
        v.kuse = kofs;
        rc = oz_gemm(S, false, v, v, n - k0, kb, reinterpret_cast<double*>(U + k0 * n + k0), n, 3, nullptr,
                     h->flag + 2, sh, 1, nullptr, OzRange(), 64);
        if (rc) return fail(rc);
      }
      const float2* Uk = (k0 > 0) ? U : nullptr;
      err = launch_potrf_blk(A, lda, k0, kb, Uk, n, LDF, LinvDF, scales, b ? w : nullptr, y, yDF, flag, sh);
      if (err != cudaSuccess) return err;
      const int64_t k1 = k0 + kb;
      if (k1 >= n) break;
      err = launch_panel_split(S, A, lda, k0, kb, k1, n, Uk, n, LinvDF + (k0 / NB) * NB * NB,
                               scales + (k0 / NB) * NB, strip, strip.e + (kofs / NB) * estride, s0, kofs, yDF,
                               b ? w : nullptr, flag, sh);
      if (err != cudaSuccess) return err;
    }
    if (s1 >= n) break;
    // bulk update of the trailing matrix, U[s1:, s1:] += L[s1:, s0:s1] L[s1:, s0:s1]^T
    OzOperand wb = oz_operand_rows(strip, S, s1 - s0);
    // (a) the next strip's columns now, on the critical path; the deferred update of strip
    //     t - 1 writes those columns too, so it must be done first
    if (t >= 1 && launchedB[t - 1] && (err = cudaStreamWaitEvent(sh, evB[t - 1], 0)) != cudaSuccess) return err;
    const int64_t nn = (n - s1 < kStrip) ? n - s1 : kStrip;
    rc = oz_gemm(S, false, wb, wb, n - s1, nn, reinterpret_cast<double*>(U + s1 * n + s1), n, 3, nullptr,
                 h->flag + 2, sh, 1, nullptr, OzRange(), 64);
    if (rc) return fail(rc);
    if ((err = cudaEventRecord(evA[t], sh)) != cudaSuccess) return err;
    // (b) the rest, U[s2:, s2:] (lower tiles), deferred to sl: it overlaps the next strip's
    //     chain, which touches only the next strip's columns
    const int64_t s2 = s1 + kStrip;
    if (s2 < n) {
      if ((err = cudaStreamWaitEvent(sl, evA[t], 0)) != cudaSuccess) return err;
      OzOperand wv = oz_operand_rows(wb, S, kStrip);
      rc = oz_gemm(S, true, wv, wv, n - s2, n - s2, reinterpret_cast<double*>(U + s2 * n + s2), n, 3, nullptr,
                   h->flag + 2, sl);
      if (rc) return fail(rc);
      if ((err = cudaEventRecord(evB[t], sl)) != cudaSuccess) return err;
      launchedB[t] = 1;
    }
  }
  // the FP64 copies of the diagonal blocks' factors for the triangular solves
  diag_to_fp64_kernel<<<(unsigned)nblk, 256, 0, sh>>>(A, lda, n, LDF, LinvDF, scales, Linv, flag);
  count_launch();
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if ((err = cudaEventRecord(e_hi, sh)) != cudaSuccess) return err;
  if ((err = cudaEventRecord(e_lo, sl)) != cudaSuccess) return err;
  if ((err = cudaStreamWaitEvent(st, e_hi, 0)) != cudaSuccess) return err;
  return cudaStreamWaitEvent(st, e_lo, 0);
}

namespace {
// backward substitution L^T x = y; w: n doubles of work space
cudaError_t backward_solve(const double* A, int64_t n, int64_t lda, const double* Linv, const double* y, double* x,
                           double* w, cudaStream_t st) {
  cudaError_t err = cudaMemcpyAsync(w, y, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (err != cudaSuccess) return err;
  const int64_t nblk = (n + NB - 1) / NB;
  for (int64_t k = nblk - 1; k >= 0; k--) {
    const int64_t k0 = k * NB;
    const int kb = (int)((n - k0) < NB ? (n - k0) : NB);
    const int64_t blocks = k0 > 0 ? (k0 + NB - 1) / NB : 1;
    bwd_step_kernel<<<(unsigned)blocks, kSolveThreads, 0, st>>>(A, lda, Linv + k * NB * NB, w, x, k0, kb);
    count_launch();
  }
  return cudaGetLastError();
}
}  // namespace

cudaError_t cholesky_solve(const double* A, int64_t n, int64_t lda, const double* Linv, const double* b, double* x,
                           double* tmp, cudaStream_t st) {
  // tmp: 2n doubles (the work vector and the forward result)
  double* w = tmp;
  double* y = tmp + n;
  cudaError_t err = cudaMemcpyAsync(w, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (err != cudaSuccess) return err;
  const int64_t nblk = (n + NB - 1) / NB;
  const int64_t cap = 2 * 152;   // two CTAs per SM of a GB300 at most: the redundant 64 x 64 product stays small
  // forward: L y = b
  for (int64_t k = 0; k < nblk; k++) {
    const int64_t k0 = k * NB;
    const int kb = (int)((n - k0) < NB ? (n - k0) : NB);
    int64_t blocks = (n - k0 - kb + 7) / 8;
    blocks = blocks < 1 ? 1 : (blocks > cap ? cap : blocks);
    fwd_step_kernel<<<(unsigned)blocks, kSolveThreads, 0, st>>>(A, lda, Linv + k * NB * NB, w, y, k0, kb, n);
    count_launch();
  }
  return backward_solve(A, n, lda, Linv, y, x, w, st);
}

cudaError_t cholesky_solve_backward(const double* A, int64_t n, int64_t lda, const double* Linv, const double* y,
                                    double* x, double* tmp, cudaStream_t st) {
  return backward_solve(A, n, lda, Linv, y, x, tmp, st);
}

}  // namespace gn
