// Vector kernels of the Gauss-Newton step: deterministic reductions (loss,
// dot products, max residual), the line-search trial point, matrix-vector
// products with J~ and G, and the damping shift G + gamma I.
// Every reduction uses a fixed grid and a fixed combination order, so the
// results are bitwise reproducible run to run.
#include <cmath>

#include "gn_internal.cuh"

namespace gn {
namespace {

constexpr int RB = 256;   // reduction blocks
constexpr int RT = 256;   // threads per reduction block

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
// max that propagates NaN (fmax would drop it)
__device__ __forceinline__ double nmax(double a, double b) { return (a != a || b != b) ? a + b : (a > b ? a : b); }
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

template <int OP>  // 0: sum x*y, 1: sum x*x, 2: max |x|
__global__ void __launch_bounds__(RT) reduce_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                    int64_t n, double* red) {
  __shared__ double s[RT / 32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)RB * RT) {
    const double a = x[i];
    if (OP == 0) acc = fma(a, y[i], acc);
    else if (OP == 1) acc = fma(a, a, acc);
    else acc = (fabs(a) > acc || a != a) ? fabs(a) : acc;
  }
  acc = (OP == 2) ? warp_max(acc) : warp_sum(acc);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < RT / 32 ? s[threadIdx.x] : 0.0;
    v = (OP == 2) ? warp_max(v) : warp_sum(v);
    if (threadIdx.x == 0) red[blockIdx.x] = v;
  }
}

// max over rows i < n of |r_i| / (w sqrt(rho_{i / ne})) (rho null: 1), NaN propagating: the
// largest unweighted residual |R_k| of the interior rows r_i = w sqrt(rho) R_k
__global__ void __launch_bounds__(RT) max_unweighted_kernel(const double* __restrict__ r,
                                                            const double* __restrict__ rho, int64_t n, int ne,
                                                            double w, double* red) {
  __shared__ double s[RT / 32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)RB * RT) {
    const double a = fabs(r[i]) / (rho ? w * sqrt(rho[i / ne]) : w);
    acc = (a > acc || a != a) ? a : acc;
  }
  acc = warp_max(acc);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < RT / 32 ? s[threadIdx.x] : 0.0;
    v = warp_max(v);
    if (threadIdx.x == 0) red[blockIdx.x] = v;
  }
}

template <int OP>
__global__ void finish_kernel(double* red, double* out) {
  __shared__ double s[RB / 32];
  double v = red[threadIdx.x];
  v = (OP == 2) ? warp_max(v) : warp_sum(v);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < RB / 32 ? s[threadIdx.x] : 0.0;
    w = (OP == 2) ? warp_max(w) : warp_sum(w);
    if (threadIdx.x == 0) *out = w;
  }
}

__global__ void axpy_trial_kernel(const double* __restrict__ theta, const double* __restrict__ delta, double alpha,
                                  int64_t P, double* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = theta[i] - alpha * delta[i];
}

// y[n] = beta*y + A^T x with A (m x n, row-major): chunks of rows give partial
// sums (coalesced over columns), summed in chunk order by gemv_t_finish.
constexpr int GEMV_CHUNKS = 64;
__global__ void gemv_t_partial(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                               const double* __restrict__ x, double* part) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (j >= n) return;
  const int64_t rows_per = (m + GEMV_CHUNKS - 1) / GEMV_CHUNKS;
  const int64_t r0 = c * rows_per, r1 = (r0 + rows_per < m) ? r0 + rows_per : m;
  double acc = 0.0;
  for (int64_t r = r0; r < r1; r++) acc = fma(A[r * lda + j], x[r], acc);
  part[(int64_t)c * n + j] = acc;
}
__global__ void gemv_t_finish(const double* __restrict__ part, int64_t n, double* y, double beta) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int c = 0; c < GEMV_CHUNKS; c++) s += part[(int64_t)c * n + j];
  y[j] = (beta != 0.0) ? fma(beta, y[j], s) : s;
}

// y[m] = beta*y + A x, one warp per row.
__global__ void gemv_n_kernel(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                              const double* __restrict__ x, double* y, double beta) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  double acc = 0.0;
  for (int64_t j = lane; j < n; j += 32) acc = fma(A[row * lda + j], x[j], acc);
  acc = warp_sum(acc);
  if (lane == 0) y[row] = (beta != 0.0) ? fma(beta, y[row], acc) : acc;
}

// G[j][i] = G[i][j] for i > j (32 x 32 tiles through shared memory).
__global__ void mirror_lower_kernel(double* G, int64_t n, int64_t ld) {
  __shared__ double tile[32][33];
  const int64_t bi = blockIdx.y, bj = blockIdx.x;   // source tile (row block bi, col block bj), bi >= bj
  if (bj > bi) return;
  const int tx = threadIdx.x, ty = threadIdx.y;     // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = bi * 32 + r, j = bj * 32 + tx;
    tile[r][tx] = (i < n && j < n) ? G[i * ld + j] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = bj * 32 + r, j = bi * 32 + tx;  // destination (row i, col j) = source (j, i)
    if (i < n && j < n && j > i) G[i * ld + j] = tile[tx][r];
  }
}

// y_i = G_ii x_i + 2 sum_{j<i} G_ij x_j from the lower triangle of a symmetric G, so that
// x . y = x^T G x (the step's model term delta^T G delta) without the upper triangle: one warp
// per row, each row's lower part read once in a fixed order (deterministic).
__global__ void quad_lower_kernel(const double* __restrict__ G, int64_t n, int64_t ld, const double* __restrict__ x,
                                  double* y) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* gr = G + row * ld;
  double s = 0.0;
  for (int64_t j = lane; j < row; j += 32) s = fma(gr[j], x[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = fma(gr[row], x[row], 2.0 * s);
}

// A = G + gamma I on the lower triangle, diagonal included: the only part the factorisations
// read (the upper triangle of A is left as it is).  One block per row, no index division; gamma
// from the device when gamma_dev is given (a captured step reads it from its state).
__global__ void copy_add_diag_kernel(const double* __restrict__ G, double* A, int64_t n, int64_t ld, double gamma,
                                     const double* __restrict__ gamma_dev) {
  const double gm = gamma_dev ? *gamma_dev : gamma;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const double* gr = G + i * ld;
    double* ar = A + i * ld;
    for (int64_t j = threadIdx.x; j <= i; j += blockDim.x) ar[j] = (j == i) ? gr[j] + gm : gr[j];
  }
}

// A[r][c] = G[r][c] (+ *gamma on the diagonal) for the columns [c0, c1) and rows r >= c of
// the lower triangle: one band of the damped matrix the factorisation reads.
__global__ void add_diag_band_kernel(const double* __restrict__ G, double* A, int64_t n, int64_t ld, int64_t c0,
                                     int64_t c1, const double* __restrict__ gamma) {
  const double gm = *gamma;
  const int64_t w = c1 - c0, total = (n - c0) * w;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = c0 + idx / w, c = c0 + idx % w;
    if (c > r) continue;
    double v = G[r * ld + c];
    if (r == c) v += gm;
    A[r * ld + c] = v;
  }
}

// G = u u^T (first) or beta G + (1 - beta) u u^T, the whole n x n matrix (row-major, ld)
__global__ void ema_rank1_kernel(double* G, int64_t n, int64_t ld, const double* __restrict__ u, double beta,
                                 int first) {
  const int64_t total = n * n;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / n, j = idx - i * n;
    const double p = u[i] * u[j];
    G[i * ld + j] = first ? p : beta * G[i * ld + j] + (1.0 - beta) * p;
  }
}

// d = alpha D + mu v (D = -delta); theta_t = theta + d[0:P); v = d (all n = P + 1 entries)
__global__ void ema_update_kernel(const double* __restrict__ theta, const double* __restrict__ delta, double* v,
                                  double alpha, double mu, int64_t P, int64_t n, double* theta_t) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = -alpha * delta[i] + mu * v[i];
    if (i < P) theta_t[i] = theta[i] + d;
    v[i] = d;
  }
}

}  // namespace

cudaError_t ema_rank1(double* G, int64_t n, int64_t ld, const double* u, double beta, int first, cudaStream_t st) {
  const int64_t total = n * n;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  ema_rank1_kernel<<<(unsigned)blocks, 256, 0, st>>>(G, n, ld, u, beta, first);
  count_launch();
  return cudaGetLastError();
}

cudaError_t ema_update(const double* theta, const double* delta, double* v, double alpha, double mu, int64_t P,
                       int64_t n, double* theta_t, cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 4) blocks = 152 * 4;
  ema_update_kernel<<<(unsigned)blocks, 256, 0, st>>>(theta, delta, v, alpha, mu, P, n, theta_t);
  count_launch();
  return cudaGetLastError();
}

cudaError_t dot_partial(const double* x, const double* y, int64_t n, double* red, cudaStream_t st) {
  reduce_kernel<0><<<RB, RT, 0, st>>>(x, y, n, red);
  count_launch();
  return cudaGetLastError();
}
cudaError_t sumsq_and_flag(const double* x, int64_t n, double* red, cudaStream_t st) {
  reduce_kernel<1><<<RB, RT, 0, st>>>(x, nullptr, n, red);
  count_launch();
  return cudaGetLastError();
}
cudaError_t finish_sum(double* red, double* out_dev, cudaStream_t st) {
  finish_kernel<0><<<1, RB, 0, st>>>(red, out_dev);
  count_launch();
  return cudaGetLastError();
}
cudaError_t max_abs_rows(const double* r, int64_t n, int stride_valid, double* red, cudaStream_t st) {
  (void)stride_valid;
  reduce_kernel<2><<<RB, RT, 0, st>>>(r, nullptr, n, red);
  count_launch();
  return cudaGetLastError();
}
cudaError_t max_abs_unweighted(const double* r, int64_t n_pts, int ne, const double* rho, double w, double* red,
                               double* out_dev, cudaStream_t st) {
  max_unweighted_kernel<<<RB, RT, 0, st>>>(r, rho, n_pts * ne, ne, w, red);
  count_launch();
  finish_kernel<2><<<1, RB, 0, st>>>(red, out_dev);
  count_launch();
  return cudaGetLastError();
}
cudaError_t finish_max(double* red, double* out_dev, cudaStream_t st) {
  finish_kernel<2><<<1, RB, 0, st>>>(red, out_dev);
  count_launch();
  return cudaGetLastError();
}
cudaError_t axpy_trial(const double* theta, const double* delta, double alpha, int64_t P, double* out,
                       cudaStream_t st) {
  int64_t blocks = (P + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  if (blocks < 1) blocks = 1;
  axpy_trial_kernel<<<(unsigned)blocks, 256, 0, st>>>(theta, delta, alpha, P, out);
  count_launch();
  return cudaGetLastError();
}
// part must hold GEMV_CHUNKS * n doubles (the caller passes the handle's scratch).
cudaError_t dgemv_t_scratch(const double* A, int64_t lda, int64_t m, int64_t n, const double* x, double* y,
                            double beta, double* part, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  dim3 g((unsigned)((n + 127) / 128), GEMV_CHUNKS);
  gemv_t_partial<<<g, 128, 0, st>>>(A, lda, m, n, x, part);
  count_launch();
  gemv_t_finish<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, n, y, beta);
  count_launch();
  return cudaGetLastError();
}
cudaError_t dgemv_n(const double* A, int64_t lda, int64_t m, int64_t n, const double* x, double* y, double beta,
                    cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const int64_t threads = m * 32;
  gemv_n_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(A, lda, m, n, x, y, beta);
  count_launch();
  return cudaGetLastError();
}
cudaError_t mirror_lower(double* G, int64_t n, int64_t ld, cudaStream_t st) {
  const int64_t nb = (n + 31) / 32;
  mirror_lower_kernel<<<dim3((unsigned)nb, (unsigned)nb), dim3(32, 8), 0, st>>>(G, n, ld);
  count_launch();
  return cudaGetLastError();
}
cudaError_t add_diag_band(const double* G, double* A, int64_t n, int64_t ld, int64_t c0, int64_t c1,
                          const double* gamma, cudaStream_t st) {
  if (c1 <= c0 || c0 >= n) return cudaSuccess;
  const int64_t total = (n - c0) * (c1 - c0);
  int64_t b = (total + 255) / 256;
  if (b > 2048) b = 2048;
  add_diag_band_kernel<<<(unsigned)b, 256, 0, st>>>(G, A, n, ld, c0, c1, gamma);
  count_launch();
  return cudaGetLastError();
}
cudaError_t quad_lower(const double* G, int64_t n, int64_t ld, const double* x, double* y, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  quad_lower_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(G, n, ld, x, y);
  count_launch();
  return cudaGetLastError();
}
cudaError_t copy_add_diag(const double* G, double* A, int64_t n, int64_t ld, double gamma, const double* gamma_dev,
                          cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  copy_add_diag_kernel<<<(unsigned)(n < 8192 ? n : 8192), 256, 0, st>>>(G, A, n, ld, gamma, gamma_dev);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gn
