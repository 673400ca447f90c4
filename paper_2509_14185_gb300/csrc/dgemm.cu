// FP64 GEMM on the DFMA pipe: the "native FP64" path of the Gram product
// G = J~^T J~ (Methods, "Second-order Optimizer"), the CCF Hilbert contraction
// J_U = K J_g, and the trailing updates of the blocked Cholesky factorisation.
//
// GB300 executes FP64 at roughly 1/60 of its FP32 rate (measured ~1.19 TFLOP/s
// DFMA), so this kernel is FP64-pipe bound for every shape used here: a
// 64x64 output tile per 256-thread block, 4x4 outputs per thread, K staged
// through shared memory 16 at a time with a register prefetch of the next
// stage.  Operand layouts are template parameters so that J~ (row-major,
// rows x P') serves as both J~^T and J~ without a transpose copy.
#include "gn_internal.cuh"

namespace gn {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <bool AK, bool BKC>
__global__ void __launch_bounds__(256) dgemm_kernel(int64_t m, int64_t n, int64_t k, double alpha,
                                                    const double* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ B, int64_t ldb, double beta,
                                                    double* C, int64_t ldc, int lower,
                                                    const double* __restrict__ rowscale) {
  const int bm = blockIdx.y, bn = blockIdx.x;
  if (lower && bn > bm) return;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int64_t m0 = (int64_t)bm * BM, n0 = (int64_t)bn * BN;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
  double ra[4], rb[4];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < 4; r++) {
      int mm, kk;
      if (AK) { kk = t & 15; mm = (t >> 4) + 16 * r; }
      else { mm = t & 63; kk = (t >> 6) + 4 * r; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      ra[r] = (gm < m && gk < k) ? (AK ? A[gm * lda + gk] : A[gk * lda + gm]) : 0.0;
      int nn, kb;
      if (BKC) { kb = t & 15; nn = (t >> 4) + 16 * r; }
      else { nn = t & 63; kb = (t >> 6) + 4 * r; }
      const int64_t gn = n0 + nn, gkb = k0 + kb;
      rb[r] = (gn < n && gkb < k) ? (BKC ? B[gn * ldb + gkb] : B[gkb * ldb + gn]) : 0.0;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int r = 0; r < 4; r++) {
      if (AK) As[t & 15][(t >> 4) + 16 * r] = ra[r];
      else As[(t >> 6) + 4 * r][t & 63] = ra[r];
      if (BKC) Bs[t & 15][(t >> 4) + 16 * r] = rb[r];
      else Bs[(t >> 6) + 4 * r][t & 63] = rb[r];
    }
  };
  load(0);
  store();
  __syncthreads();
  for (int64_t k0 = 0; k0 < k; k0 += BK) {
    const bool more = k0 + BK < k;
    if (more) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; kk++) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
    if (more) {
      store();
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int64_t r = m0 + ty + 16 * i;
    if (r >= m) continue;
    const double rs = rowscale ? rowscale[r] * alpha : alpha;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int64_t c = n0 + tx + 16 * j;
      if (c >= n) continue;
      double v = rs * acc[i][j];
      if (beta != 0.0) v = fma(beta, C[r * ldc + c], v);
      C[r * ldc + c] = v;
    }
  }
}

}  // namespace

cudaError_t dgemm(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda, bool a_kcontig,
                  const double* B, int64_t ldb, bool b_kcontig, double beta, double* C, int64_t ldc, bool lower,
                  const double* rowscale, cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  const int64_t gm = (m + BM - 1) / BM, gn = (n + BN - 1) / BN;
  if (gm > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)gn, (unsigned)gm);
  // k <= 0 is valid: the kernel then only applies C = beta C
  if (a_kcontig && b_kcontig)
    dgemm_kernel<true, true><<<grid, 256, 0, st>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, lower, rowscale);
  else if (a_kcontig && !b_kcontig)
    dgemm_kernel<true, false><<<grid, 256, 0, st>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, lower, rowscale);
  else if (!a_kcontig && b_kcontig)
    dgemm_kernel<false, true><<<grid, 256, 0, st>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, lower, rowscale);
  else
    dgemm_kernel<false, false><<<grid, 256, 0, st>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, lower, rowscale);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gn
