// Discrete Hilbert operator of the CCF velocity U = H Theta.
//
// The paper names the CCF equation (Results) but leaves its discretisation to
// the Supplementary Information.  This library's reading: with
// Theta(s) = s g(s), U(x) = x H[g](x); on the circle s = tan(psi/2) the
// transform is the periodic conjugate function minus a constant, taken by the
// M-point trapezoid rule on psi_j = -pi + (j + 1/2) 2pi/M with the principal
// value removed by subtracting g(x):
//   U_i = (x_i/M) [ sum_j (g_j - g_i) cot((phi_i - psi_j)/2) - sum_j g_j s_j ]
//       = sum_j K_ij g_j + D_i g_i,
//   K_ij = (x_i/M)(cot_ij - s_j),  D_i = -(x_i/M) sum_j cot_ij.
// g is odd and the nodes come in pairs s_{M-1-j} = -s_j, so the library keeps
// only the M/2 positive nodes and the folded matrix
//   Kf_ij' = K_{i, M/2+j'} - K_{i, M/2-1-j'}.
#include <cmath>

#include "gn_internal.cuh"

namespace gn {
namespace {

__device__ __forceinline__ double node_psi(int j, int M) {
  return -M_PI + (j + 0.5) * (2.0 * M_PI / M);
}

// One warp per point: the folded row of K and the diagonal coefficient D_i.
__global__ void hilbert_build_kernel(const double* __restrict__ y, int64_t n, int M, double* kf, double* dcoef,
                                     double* snode) {
  const int Mh = M / 2;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid == 0) {
    for (int jp = lane; jp < Mh; jp += 32) snode[jp] = tan(0.5 * node_psi(Mh + jp, M));
  }
  if (wid >= n) return;
  const double x = y[wid];
  const double phi = 2.0 * atan(x);
  const double xm = x / M;
  double csum = 0.0;
  for (int jp = lane; jp < Mh; jp += 32) {
    const int jpos = Mh + jp, jneg = Mh - 1 - jp;
    const double pp = node_psi(jpos, M), pn = node_psi(jneg, M);
    const double sp = tan(0.5 * pp), sn = tan(0.5 * pn);
    const double cp = 1.0 / tan(0.5 * (phi - pp));
    const double cn = 1.0 / tan(0.5 * (phi - pn));
    kf[wid * Mh + jp] = xm * ((cp - sp) - (cn - sn));
    csum += cp + cn;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) csum += __shfl_down_sync(0xffffffffu, csum, o);
  if (lane == 0) dcoef[wid] = -xm * csum;
}

// The same operator as a Taylor series in the collocation point x (for the derivative-loss
// rows): with x = tan(phi/2) and s_j = tan(psi_j/2) the kernel is rational in x,
// cot((phi - psi_j)/2) = (1 + x s_j) / (x - s_j), whose coefficients in dx = x - x0 follow from
// 1 / (t + dx) = sum_k (-1)^k dx^k / t^(k+1), t = x0 - s_j.  Then
//   K_j(x) = (x/M)(cot_j(x) - s_j),  D(x) = -(x/M) sum_j cot_j(x)
// (the factor x = x0 + dx shifts the coefficients by one).  One warp per point; the folded
// pair (M/2 + j', M/2 - 1 - j') as in hilbert_build_kernel.  kOrdMax bounds the order.
constexpr int kOrdMax = 4;
__device__ __forceinline__ void cot_series(double x0, double s, int order, double* c) {
  const double t = x0 - s;
  const double it = 1.0 / t;
  double r[kOrdMax + 1];
  double pw = it;
#pragma unroll
  for (int k = 0; k <= kOrdMax; k++) {
    r[k] = (k & 1) ? -pw : pw;   // (-1)^k / t^(k+1)
    pw *= it;
  }
  const double a = 1.0 + x0 * s;
#pragma unroll
  for (int m = 0; m <= kOrdMax; m++) c[m] = (m <= order) ? a * r[m] + (m > 0 ? s * r[m - 1] : 0.0) : 0.0;
}

__global__ void hilbert_series_kernel(const double* __restrict__ y, int64_t n, int M, int order, double* kd,
                                      double* dd) {
  const int Mh = M / 2;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= n) return;
  const double x0 = y[wid];
  double csum[kOrdMax + 1];
#pragma unroll
  for (int m = 0; m <= kOrdMax; m++) csum[m] = 0.0;
  for (int jp = lane; jp < Mh; jp += 32) {
    const int jpos = Mh + jp, jneg = Mh - 1 - jp;
    const double sp = tan(0.5 * node_psi(jpos, M)), sn = tan(0.5 * node_psi(jneg, M));
    double cp[kOrdMax + 1], cn[kOrdMax + 1];
    cot_series(x0, sp, order, cp);
    cot_series(x0, sn, order, cn);
    // K coefficients: (x0 c'_m + c'_{m-1}) / M with c' = cot - s (the constant term only)
    double prev = 0.0;
#pragma unroll
    for (int m = 0; m <= kOrdMax; m++) {
      if (m > order) break;
      const double fp = cp[m] - (m == 0 ? sp : 0.0), fn = cn[m] - (m == 0 ? sn : 0.0);
      const double cur = fp - fn;                       // the folded pair
      kd[((int64_t)m * n + wid) * Mh + jp] = (x0 * cur + prev) / M;
      prev = cur;
      csum[m] += cp[m] + cn[m];
    }
  }
#pragma unroll
  for (int m = 0; m <= kOrdMax; m++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) csum[m] += __shfl_down_sync(0xffffffffu, csum[m], o);
  if (lane == 0) {
    double prev = 0.0;
    for (int m = 0; m <= order; m++) {
      dd[(int64_t)m * n + wid] = -(x0 * csum[m] + prev) / M;
      prev = csum[m];
    }
  }
}

}  // namespace

cudaError_t hilbert_series_build(const double* y, int64_t n, int M, int order, double* kd, double* dd,
                                 cudaStream_t st) {
  if (order < 0 || order > kOrdMax) return cudaErrorInvalidValue;
  if (n == 0) return cudaSuccess;
  const int64_t threads = n * 32;
  hilbert_series_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(y, n, M, order, kd, dd);
  count_launch();
  return cudaGetLastError();
}

cudaError_t hilbert_build(const double* y, int64_t n, int M, double* kf, double* dcoef, double* snode,
                          cudaStream_t st) {
  const int64_t warps = n > 0 ? n : 1;
  const int64_t threads = warps * 32;
  hilbert_build_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(y, n, M, kf, dcoef, snode);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gn
