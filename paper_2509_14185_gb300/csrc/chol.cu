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
  __shared__ double rinv;
  for (int j = 0; j < kb; j++) {
    if (t == 0) {
      const double d = S[j][j];
      if (!(d > 0.0) || !isfinite(d)) bad = 1;
      const double piv = sqrt(d);
      S[j][j] = piv;
      rinv = 1.0 / piv;   // one division per column; the column is scaled by multiplication
    }
    __syncthreads();
    if (bad) break;
    const double r = rinv;
    for (int i = j + 1 + t; i < kb; i += blockDim.x) S[i][j] *= r;
    __syncthreads();
    // trailing update of the lower triangle of the diagonal block (lower pairs only)
    const int rem = kb - j - 1;
    const int npair = rem * (rem + 1) / 2;
    for (int idx = t; idx < npair; idx += blockDim.x) {
      // idx -> (a, b) with 0 <= b <= a < rem, row-major over the lower triangle
      int a = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
      while ((a + 1) * (a + 2) / 2 <= idx) a++;
      while (a * (a + 1) / 2 > idx) a--;
      const int b = idx - a * (a + 1) / 2;
      const int i = j + 1 + a, c = j + 1 + b;
      S[i][c] = fma(-S[i][j], S[c][j], S[i][c]);
    }
    __syncthreads();
  }
  if (bad) {
    if (t == 0) atomicExch(flag, 1);
    return;
  }
  // inverse of the lower-triangular factor:
  // X[c][c] = 1/L[c][c], X[i][c] = -(sum_{q=c}^{i-1} L[i][q] X[q][c]) / L[i][i].
  // Dependent FP64 operations are slow on this part, so each column's dot
  // products are split over 4 threads (lanes 4c .. 4c+3 of one warp) and the
  // reciprocals of the pivots are formed once, in parallel.
  if (t < kb) xd[t] = 1.0 / S[t][t];
  __syncthreads();
  {
    const int c = t >> 2, part = t & 3;
    for (int i = 1; i < NB; i++) {   // uniform trip count: the shuffles need the whole warp
      const bool act = (c < kb && i < kb && i > c);
      double s = 0.0;
      if (act) {
        if (part == 0) s = S[i][c] * xd[c];
        for (int q = c + 1 + part; q < i; q += 4) s = fma(S[i][q], S[c][q], s);
      }
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (act && part == 0) S[c][i] = -s * xd[i];
      __syncwarp();
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

// A[i][j] -= U[i][j] (double-FP32 -> FP64) for the panel columns j in [k0, k0+kb), rows i >= j
__global__ void panel_fix_kernel(double* A, int64_t lda, const float2* __restrict__ U, int64_t ldu, int64_t k0,
                                 int kb, int64_t n) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = k0 + idx / kb, j = k0 + idx % kb;
  if (i >= n || j > i) return;
  const float2 u = U[i * ldu + j];
  A[i * lda + j] -= (double)u.x + (double)u.y;
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
  // Workspace: the L21 operand, the Linv operand, and U, the double-FP32 sum of
  // all trailing updates L21 L21^T so far (n x n float2).  U is accumulated on
  // the FP32 pipe by the split GEMM's epilogue; only the 64 columns about to be
  // factored are converted and applied in FP64 (panel_fix), so the FP64 work of
  // the trailing updates drops from O(n^3/64) to O(n^2).
  cudaStream_t st = h->st;
  *rc_out = GN_OK;
  const size_t opb = oz_operand_bytes(S, n, NB), opi = oz_operand_bytes(S, NB, NB);
  const size_t ub = ((size_t)n * n * sizeof(float2) + 255) / 256 * 256;
  int rc = ensure_split_ws(h, ub + opb + opi + 1024);
  if (rc) {
    *rc_out = rc;
    return cudaErrorMemoryAllocation;
  }
  unsigned char* base = static_cast<unsigned char*>(h->split_ws);
  float2* U = reinterpret_cast<float2*>(base);
  cudaError_t err = cudaMemsetAsync(U, 0, (size_t)n * n * sizeof(float2), st);
  if (err != cudaSuccess) return err;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int kb = (int)((n - k0) < NB ? (n - k0) : NB);
    if (k0 > 0) {
      const int64_t cnt = (n - k0) * kb;
      panel_fix_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(A, lda, U, n, k0, kb, n);
      count_launch();
    }
    potrf_diag_kernel<<<1, 256, 0, st>>>(A, lda, k0, kb, Linv, flag);
    count_launch();
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const int64_t k1 = k0 + kb;
    if (k1 >= n) break;
    double* Lk = Linv + (k0 / NB) * NB * NB;
    // panel solve L21 = A21 Linv^T as a split GEMM (A21's slices are taken before it is overwritten)
    OzOperand L = oz_operand_at(base + ub, S, n - k1, kb);
    OzOperand I = oz_operand_at(base + ub + opb, S, kb, kb);
    rc = oz_prepare_rows(S, A + k1 * lda + k0, lda, n - k1, kb, L, st);
    if (!rc) rc = oz_prepare_rows(S, Lk, NB, kb, kb, I, st);
    if (!rc) rc = oz_gemm(S, false, L, I, n - k1, kb, A + k1 * lda + k0, lda, 0, nullptr, h->flag + 2, st);
    // trailing update U[k1:, k1:] += L21 L21^T (double-FP32, FP32 pipe)
    if (!rc) rc = oz_prepare_rows(S, A + k1 * lda + k0, lda, n - k1, kb, L, st);
    if (!rc)
      rc = oz_gemm(S, true, L, L, n - k1, n - k1, reinterpret_cast<double*>(U + k1 * n + k1), n, 3, nullptr,
                   h->flag + 2, st);
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
