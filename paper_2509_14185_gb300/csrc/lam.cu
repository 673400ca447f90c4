// Strategies for the blow-up rate lambda (Methods, "Identifying Admissible
// lambda Values"): training at a fixed lambda, the lambda-inference rule at the
// origin (item 2) and the pieces of funnel inference (item 3): the signed
// residual of largest magnitude near the origin and the secant update.
//
// lambda-inference rules (the paper prints the Boussinesq one; the others follow
// from the same steps on this library's residual operators):
//   Boussinesq  lambda = -3 - 2 d1 U1(0,0),   IPM  lambda = -2 - 2 d1 U1(0,0),
//   with U1 = d2 Psi, so d1 U1 = d12 Psi;     CCF  lambda = -2 - 2 U'(0).
// For CCF, U = x H[g] with g = Theta / x, so U'(0) = H[g](0).  The discrete
// operator at x = 0 (phi = 0, g(0) = 0) over the node pairs s_j, -s_j is
//   H[g](0) = (1/M) sum_j g_j (cot(-psi_j / 2) - s_j) = -(2/M) sum_{s_j > 0} g_j (s_j + 1/s_j).
#include <cmath>
#include <cstring>

#include "gn_internal.cuh"

namespace gn {
namespace {

#define GN_L_TRY(x)                                         \
  do {                                                      \
    cudaError_t e_ = GN_NOTE(x);                            \
    if (e_ != cudaSuccess) return GN_ERR_CUDA;              \
  } while (0)

constexpr int kRedThreads = 256;

// out = -(2/M) sum_j g_j (s_j + 1/s_j) over the positive nodes (one block, fixed order)
__global__ void __launch_bounds__(kRedThreads) ccf_du0_kernel(const double* __restrict__ g,
                                                              const double* __restrict__ s, int Mh, int M,
                                                              double* out) {
  __shared__ double part[kRedThreads];
  double acc = 0.0;
  for (int j = threadIdx.x; j < Mh; j += kRedThreads) acc += g[j] * (s[j] + 1.0 / s[j]);
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = -(2.0 / M) * part[0];
}

// The interior residual of largest |R| among the points with |y| <= radius, with its sign.
// Rows are point-major (row i NE + k); ties go to the smaller row, i.e. the first point, then
// the first equation.  out[0] = value (0 if no point), out[1] = point index (-1 if none).
__global__ void __launch_bounds__(1024) signed_max_kernel(const double* __restrict__ r, const double* __restrict__ y,
                                                          int64_t n, int d, int ne, double radius, double* out) {
  __shared__ double sv[1024];
  __shared__ double sa[1024];
  __shared__ long long si[1024];
  double bv = 0.0, ba = -1.0;
  long long bi = -1;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    // |y| as sqrt(y1 y1 + y2 y2) with separately rounded products (no contraction)
    double rr = __dmul_rn(y[i], y[i]);
    if (d == 2) rr = __dadd_rn(rr, __dmul_rn(y[n + i], y[n + i]));
    if (!(sqrt(rr) <= radius)) continue;
    for (int k = 0; k < ne; k++) {
      const double v = r[i * ne + k];
      const double a = fabs(v);
      if (a > ba) {   // rows visited in increasing order per thread: keeps the first on ties
        ba = a;
        bv = v;
        bi = i * ne + k;
      }
    }
  }
  sv[threadIdx.x] = bv;
  sa[threadIdx.x] = ba;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      const int o = threadIdx.x + w;
      const bool take = sa[o] > sa[threadIdx.x] || (sa[o] == sa[threadIdx.x] && si[o] >= 0 &&
                                                     (si[threadIdx.x] < 0 || si[o] < si[threadIdx.x]));
      if (take) {
        sa[threadIdx.x] = sa[o];
        sv[threadIdx.x] = sv[o];
        si[threadIdx.x] = si[o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = si[0] >= 0 ? sv[0] : 0.0;
    out[1] = si[0] >= 0 ? (double)(si[0] / ne) : -1.0;
  }
}

}  // namespace
}  // namespace gn

using namespace gn;

extern "C" {

int gn_set_lambda_trainable(gn_handle* h, int trainable) {
  if (!h || (trainable != 0 && trainable != 1)) return GN_ERR_INVALID;
  h->lam_frozen = trainable ? 0 : 1;
  return GN_OK;
}

int gn_lambda_inference(gn_handle* h, const double* theta, double lambda, double* lambda_out) {
  if (!h || !theta || !lambda_out) return GN_ERR_INVALID;
  if (h->eq == GN_BURGERS) {
    set_detail(__FILE__, __LINE__, "Burgers: U'(0) = -1 for every lambda, no lambda-inference rule");
    return GN_ERR_UNSUPPORTED;
  }
  cudaStream_t st = h->st;
  GN_L_TRY(launch_transpose_weights(h->net, theta, h->wt, st));
  JetArgs a;
  memset(&a, 0, sizeof(a));
  a.net = h->net;
  a.eq = h->eq;
  a.theta = theta;
  a.wt = h->wt;
  a.fW = h->fourierW;
  a.lam = lambda;
  a.flag = h->flag;
  a.mode = MODE_RESIDUAL;
  double* slot = h->red + 560;
  if (h->eq == GN_CCF) {
    // g at the positive nodes, then H[g](0)
    a.kind = KIND_NODE;
    a.n = h->Mh;
    a.y = h->snode;
    a.ystride = h->Mh;
    a.wscale = 1.0;
    a.r = h->gnode;
    GN_L_TRY(launch_jet(a, st, nullptr));
    ccf_du0_kernel<<<1, kRedThreads, 0, st>>>(h->gnode, h->snode, h->Mh, h->M, slot);
    count_launch();
    GN_L_TRY(cudaGetLastError());
  } else {
    // field jets at the origin; d12 Psi is the Hessian's middle entry of the last field
    double* y0 = h->red + 520;
    GN_L_TRY(cudaMemsetAsync(y0, 0, 2 * sizeof(double), st));
    a.kind = KIND_PROBE;
    a.n = 1;
    a.y = y0;
    a.ystride = 1;
    a.wscale = 1.0;
    a.r = h->red + 530;   // NF x 6 values
    GN_L_TRY(launch_jet(a, st, nullptr));
    GN_L_TRY(cudaMemcpyAsync(slot, h->red + 530 + (h->nf - 1) * 6 + 4, sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  GN_L_TRY(cudaMemcpyAsync(h->hpin + 40, slot, sizeof(double), cudaMemcpyDeviceToHost, st));
  GN_L_TRY(cudaStreamSynchronize(st));
  const double v = h->hpin[40];   // CCF: U'(0); 2D: d1 U1(0, 0) = d12 Psi(0, 0)
  const double base = h->eq == GN_BOUSSINESQ ? -3.0 : -2.0;
  *lambda_out = base - 2.0 * v;
  return std::isfinite(*lambda_out) ? GN_OK : GN_ERR_NONFINITE;
}

int gn_signed_max_residual(gn_handle* h, const double* theta, double lambda, double radius, double* r_hat,
                           int64_t* point) {
  if (!h || !theta || !r_hat || !(radius >= 0.0)) return GN_ERR_INVALID;
  if (h->p.n_pts == 0) {
    *r_hat = 0.0;
    if (point) *point = -1;
    return GN_OK;
  }
  Pass ps = {MODE_RESIDUAL, h->r, nullptr, 0, 0, 0, nullptr};
  ps.unweighted = true;
  int rc = run_pass(h, theta, lambda, ps, nullptr);
  if (rc) return rc;
  double* slot = h->red + 570;
  signed_max_kernel<<<1, 1024, 0, h->st>>>(h->r, h->p.y, h->p.n_pts, h->d, h->ne, radius, slot);
  count_launch();
  GN_L_TRY(cudaGetLastError());
  GN_L_TRY(cudaMemcpyAsync(h->hpin + 42, slot, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  GN_L_TRY(cudaStreamSynchronize(h->st));
  *r_hat = h->hpin[42];
  if (point) *point = (int64_t)h->hpin[43];
  return GN_OK;
}

int gn_field_jets(gn_handle* h, const double* theta, double lambda, const double* y, int64_t n, double* out) {
  if (!h || !theta || !out || n < 0 || (n > 0 && !y)) return GN_ERR_INVALID;
  if (n == 0) return GN_OK;
  cudaStream_t st = h->st;
  GN_L_TRY(launch_transpose_weights(h->net, theta, h->wt, st));
  JetArgs a;
  memset(&a, 0, sizeof(a));
  a.net = h->net;
  a.eq = h->eq;
  a.theta = theta;
  a.wt = h->wt;
  a.fW = h->fourierW;
  a.lam = lambda;
  a.flag = h->flag;
  a.mode = MODE_RESIDUAL;
  a.kind = KIND_PROBE;
  a.n = n;
  a.y = y;
  a.ystride = n;
  a.wscale = 1.0;
  a.r = out;
  GN_L_TRY(launch_jet(a, st, nullptr));
  return GN_OK;
}

int gn_field_jets_ld(const gn_handle* h, int64_t* ld) {
  if (!h || !ld) return GN_ERR_INVALID;
  *ld = probe_ld(h->eq, h->d, h->nf);
  return GN_OK;
}

int gn_funnel_next(const double* lambdas, const double* r_hats, int n, double dlambda, double* lambda_next) {
  if (!lambdas || !r_hats || !lambda_next || n < 1) return GN_ERR_INVALID;
  if (n == 1) {
    *lambda_next = lambdas[0] + dlambda;
    return GN_OK;
  }
  const double l0 = lambdas[n - 2], l1 = lambdas[n - 1], r0 = r_hats[n - 2], r1 = r_hats[n - 1];
  if (r1 == r0) return GN_ERR_INVALID;
  *lambda_next = l1 - r1 * (l1 - l0) / (r1 - r0);
  return GN_OK;
}

}  // extern "C"
