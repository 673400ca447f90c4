// Damped FP64 Cholesky solve (G + gamma I) delta = g of the Gauss-Newton step
// (Methods, "Second-order Optimizer").
//
// Blocked right-looking factorisation on a row-major matrix, lower triangle,
// block size 64:
//   1. one CTA factors the 64 x 64 diagonal block in shared memory and also
//      forms its inverse Linv_k (kept for the triangular solves);
//   2. the panel below it is solved as a GEMM, L21 = A21 Linv_k^T;
//   3. the trailing matrix is updated A22 -= L21 L21^T (lower tiles only).
// A non-positive pivot sets a device flag; later blocks skip their work and
// the host escalates the damping.  The triangular solves use the stored
// diagonal inverses: a tiny 64 x 64 product per block plus a GEMV of the
// remaining vector spread over all SMs.
#include <cmath>

#include "gn_internal.cuh"

namespace gn {
namespace {

constexpr int NB = kCholNB;

__global__ void __launch_bounds__(256) potrf_diag_kernel(double* A, int64_t lda, int64_t k0, int kb, double* Linv,
                                                         int* flag) {
  // S: the factor in the lower triangle; the inverse's strict lower part is
  // kept transposed in S's strict upper triangle and its diagonal in xd.
  __shared__ double S[NB][NB + 1];
  __shared__ double xd[NB];
  __shared__ int bad;
  if (*flag) return;
  const int t = threadIdx.x;
  if (t == 0) bad = 0;
  for (int idx = t; idx < NB * NB; idx += blockDim.x) {
    const int i = idx / NB, j = idx % NB;
    S[i][j] = (i < kb && j < kb && j <= i) ? A[(k0 + i) * lda + k0 + j] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < kb; j++) {
    if (t == 0) {
      const double d = S[j][j];
      if (!(d > 0.0) || !isfinite(d)) bad = 1;
      S[j][j] = sqrt(d);
    }
    __syncthreads();
    if (bad) break;
    const double piv = S[j][j];
    for (int i = j + 1 + t; i < kb; i += blockDim.x) S[i][j] /= piv;
    __syncthreads();
    // trailing update of the lower triangle of the diagonal block
    const int rem = kb - j - 1;
    for (int idx = t; idx < rem * rem; idx += blockDim.x) {
      const int i = j + 1 + idx / rem, c = j + 1 + idx % rem;
      if (c <= i) S[i][c] -= S[i][j] * S[c][j];
    }
    __syncthreads();
  }
  if (bad) {
    if (t == 0) atomicExch(flag, 1);
    return;
  }
  // inverse of the lower-triangular factor, one column c per thread:
  // X[c][c] = 1/L[c][c], X[i][c] = -(sum_{q=c}^{i-1} L[i][q] X[q][c]) / L[i][i]
  if (t < kb) {
    const int c = t;
    xd[c] = 1.0 / S[c][c];
    for (int i = c + 1; i < kb; i++) {
      double s = S[i][c] * xd[c];
      for (int q = c + 1; q < i; q++) s = fma(S[i][q], S[c][q], s);
      S[c][i] = -s / S[i][i];
    }
  }
  __syncthreads();
  double* Lk = Linv + (k0 / NB) * NB * NB;
  for (int idx = t; idx < NB * NB; idx += blockDim.x) {
    const int i = idx / NB, j = idx % NB;
    if (i < kb && j < kb && j <= i) A[(k0 + i) * lda + k0 + j] = S[i][j];
    double x = 0.0;
    if (i < kb && j < kb) x = (i == j) ? xd[i] : (i > j ? S[j][i] : 0.0);
    Lk[idx] = x;
  }
}

// x_k = Linv_k v_k (trans = 0) or Linv_k^T v_k (trans = 1), in place on v[k0 .. k0+kb)
__global__ void tri_block_kernel(const double* __restrict__ Lk, double* v, int64_t k0, int kb, int trans) {
  __shared__ double s[NB];
  const int i = threadIdx.x;
  if (i < kb) s[i] = v[k0 + i];
  __syncthreads();
  if (i < kb) {
    double acc = 0.0;
    if (!trans) {
      for (int q = 0; q <= i; q++) acc = fma(Lk[i * NB + q], s[q], acc);
    } else {
      for (int q = i; q < kb; q++) acc = fma(Lk[q * NB + i], s[q], acc);
    }
    v[k0 + i] = acc;
  }
}

// forward update: v[k1 + r] -= sum_t L[k1 + r][k0 + t] v[k0 + t], one warp per row
__global__ void fwd_update_kernel(const double* __restrict__ L, int64_t lda, double* v, int64_t k0, int kb,
                                  int64_t k1, int64_t n) {
  const int64_t row = k1 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double acc = 0.0;
  for (int q = lane; q < kb; q += 32) acc = fma(L[row * lda + k0 + q], v[k0 + q], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) v[row] -= acc;
}

// backward update: v[j] -= sum_t L[k0 + t][j] v[k0 + t] for j < k0 (coalesced over j)
__global__ void bwd_update_kernel(const double* __restrict__ L, int64_t lda, double* v, int64_t k0, int kb) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k0) return;
  double acc = 0.0;
  for (int q = 0; q < kb; q++) acc = fma(L[(k0 + q) * lda + j], v[k0 + q], acc);
  v[j] -= acc;
}

}  // namespace

cudaError_t cholesky_factor(double* A, int64_t n, int64_t lda, double* Linv, int* flag, cudaStream_t st) {
  cudaError_t err = cudaSuccess;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int kb = (int)((n - k0) < NB ? (n - k0) : NB);
    potrf_diag_kernel<<<1, 256, 0, st>>>(A, lda, k0, kb, Linv, flag);
    count_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const int64_t k1 = k0 + kb;
    if (k1 >= n) break;
    const double* Lk = Linv + (k0 / NB) * NB * NB;
    // panel: A21 <- A21 Linv_k^T   (C(i,j) = sum_t A21[i][t] Linv_k[j][t])
    err = dgemm(n - k1, kb, kb, 1.0, A + k1 * lda + k0, lda, true, Lk, NB, true, 0.0, A + k1 * lda + k0, lda,
                false, nullptr, st);
    if (err != cudaSuccess) return err;
    // trailing: A22 -= L21 L21^T (lower)
    err = dgemm(n - k1, n - k1, kb, -1.0, A + k1 * lda + k0, lda, true, A + k1 * lda + k0, lda, true, 1.0,
                A + k1 * lda + k1, lda, true, nullptr, st);
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

// Same blocked factorisation with the trailing update A22 -= L21 L21^T on the
// tensor cores (split GEMM, S slices): the diagonal blocks and the panel solve
// stay FP64; the bulk (P'^3/3 of the work) becomes BF16 slice products with
// exact level accumulation.  *rc_out receives a GN_ERR_* code on failure.
cudaError_t cholesky_factor_split(gn_handle* h, double* A, int64_t n, int64_t lda, double* Linv, int* flag, int S,
                                  int* rc_out) {
  cudaStream_t st = h->st;
  *rc_out = GN_OK;
  const size_t opb = oz_operand_bytes(S, n, NB);
  int rc = ensure_split_ws(h, opb + 256);
  if (rc) {
    *rc_out = rc;
    return cudaErrorMemoryAllocation;
  }
  cudaError_t err = cudaSuccess;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int kb = (int)((n - k0) < NB ? (n - k0) : NB);
    potrf_diag_kernel<<<1, 256, 0, st>>>(A, lda, k0, kb, Linv, flag);
    count_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const int64_t k1 = k0 + kb;
    if (k1 >= n) break;
    const double* Lk = Linv + (k0 / NB) * NB * NB;
    err = dgemm(n - k1, kb, kb, 1.0, A + k1 * lda + k0, lda, true, Lk, NB, true, 0.0, A + k1 * lda + k0, lda,
                false, nullptr, st);
    if (err != cudaSuccess) return err;
    OzOperand L = oz_operand_at(h->split_ws, S, n - k1, kb);
    rc = oz_prepare_rows(S, A + k1 * lda + k0, lda, n - k1, kb, L, st);
    if (!rc) rc = oz_gemm(S, true, L, L, n - k1, n - k1, A + k1 * lda + k1, lda, 2, nullptr, h->flag + 2, st);
    if (rc) {
      *rc_out = rc;
      return cudaErrorUnknown;
    }
  }
  return cudaSuccess;
}

cudaError_t cholesky_solve(const double* A, int64_t n, int64_t lda, const double* Linv, const double* b, double* x,
                           double* tmp, cudaStream_t st) {
  (void)tmp;
  cudaError_t err = cudaMemcpyAsync(x, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (err != cudaSuccess) return err;
  const int64_t nblk = (n + NB - 1) / NB;
  // forward: L z = b
  for (int64_t k = 0; k < nblk; k++) {
    const int64_t k0 = k * NB;
    const int kb = (int)((n - k0) < NB ? (n - k0) : NB);
    tri_block_kernel<<<1, NB, 0, st>>>(Linv + k * NB * NB, x, k0, kb, 0);
    count_launch();
    const int64_t k1 = k0 + kb;
    if (k1 < n) {
      const int64_t threads = (n - k1) * 32;
      fwd_update_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(A, lda, x, k0, kb, k1, n);
      count_launch();
    }
  }
  // backward: L^T x = z
  for (int64_t k = nblk - 1; k >= 0; k--) {
    const int64_t k0 = k * NB;
    const int kb = (int)((n - k0) < NB ? (n - k0) : NB);
    tri_block_kernel<<<1, NB, 0, st>>>(Linv + k * NB * NB, x, k0, kb, 1);
    count_launch();
    if (k0 > 0) bwd_update_kernel<<<(unsigned)((k0 + 255) / 256), 256, 0, st>>>(A, lda, x, k0, kb);
    count_launch();
  }
  return cudaGetLastError();
}

}  // namespace gn
