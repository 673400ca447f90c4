// Multi-stage training (Methods, "Multi-stage Training"): a second network learns
// the error of the first.  With Phi_exact = Phi_1 + eps Phi_2, the stage-2 problem
// of a handle has the fields Phi_1 + eps Phi_2, Phi_1 the frozen stage-1 network and
// Phi_2 the handle's own network, every row divided by eps (the normalised stage-2
// equation R(Phi_1 + eps Phi_2) / eps = R_1 / eps + D[Phi_1] Phi_2 + O(eps)), and
// lambda held fixed.  The residual of the composed field is kept in full (the paper
// drops its O(eps^2) part, which lies below FP64 resolution of the rows for the eps
// of a converged first stage).
//
// Phi_1 does not change during stage 2, so its jets (value, gradient, Hessian per
// field, and g = Theta / y for CCF) are evaluated once at every point of the handle
// by the jet kernel's probe mode and kept; the kernels then only add eps Phi_2.
#include <cmath>
#include <cstring>

#include "gn_internal.cuh"

using namespace gn;

namespace {

#define GN_S_TRY(x)                                         \
  do {                                                      \
    cudaError_t e_ = GN_NOTE(x);                            \
    if (e_ != cudaSuccess) {                                \
      rc = GN_ERR_CUDA;                                     \
      goto done;                                            \
    }                                                       \
  } while (0)

}  // namespace

extern "C" {

int gn_set_stage1(gn_handle* h, int n_layers1, const int* widths1, const double* theta1, double lambda, double eps) {
  if (!h || !widths1 || !theta1 || n_layers1 < 1 || n_layers1 > GN_MAX_LAYERS) return GN_ERR_INVALID;
  if (!(eps > 0.0) || !std::isfinite(eps) || !std::isfinite(lambda)) return GN_ERR_INVALID;
  if (widths1[0] != h->d || widths1[n_layers1] != h->nf) return GN_ERR_INVALID;
  if (h->p.n_d1 > 0 || h->p.n_d2 > 0) {   // the derivative rows' kernel has no second stage
    set_detail(__FILE__, __LINE__, "derivative-loss rows with a second stage");
    return GN_ERR_UNSUPPORTED;
  }
  for (int l = 1; l < n_layers1; l++)
    if (widths1[l] < 1 || widths1[l] > 256) return GN_ERR_INVALID;
  // the stage-1 network's layout (as gn_init lays out theta)
  NetDesc net1;
  memset(&net1, 0, sizeof(net1));
  net1.L = n_layers1;
  net1.exp_out = h->net.exp_out;   // stage 1 was trained with the handle's output map
  net1.maxw = 2;
  for (int l = 0; l <= n_layers1; l++) {
    net1.w[l] = widths1[l];
    if (widths1[l] > net1.maxw) net1.maxw = widths1[l];
  }
  int64_t off = 0, offT = 0;
  for (int l = 0; l < n_layers1; l++) {
    net1.offW[l] = off;
    net1.offT[l] = offT;
    off += (int64_t)net1.w[l] * net1.w[l + 1];
    offT += (int64_t)net1.w[l] * net1.w[l + 1];
    net1.offB[l] = off;
    off += net1.w[l + 1];
  }
  net1.P = off;

  const int64_t ld = probe_ld(h->eq, h->d, h->nf);
  cudaStream_t st = h->st;
  double* wt1 = nullptr;
  int rc = GN_OK;
  {
    if (GN_NOTE(cudaMalloc((void**)&wt1, (size_t)net1.P * sizeof(double))) != cudaSuccess) return GN_ERR_OOM;
    auto grow = [&](double** p, int64_t count) -> bool {
      if (*p) return true;
      return GN_NOTE(cudaMalloc((void**)p, (size_t)(count > 0 ? count : 1) * sizeof(double))) == cudaSuccess;
    };
    if (!grow(&h->base_int, h->p.n_pts * ld) || !grow(&h->base_wall, h->p.n_bnd * ld) || !grow(&h->base_norm, ld) ||
        !grow(&h->base_inf, h->p.n_inf * ld) || !grow(&h->base_relu, h->p.n_relu * ld) ||
        (h->eq == GN_CCF && !grow(&h->base_node, h->Mh))) {
      cudaFree(wt1);
      return GN_ERR_OOM;
    }
    GN_S_TRY(launch_transpose_weights(net1, theta1, wt1, st));
    JetArgs a;
    memset(&a, 0, sizeof(a));
    a.net = net1;
    a.eq = h->eq;
    a.mode = MODE_RESIDUAL;
    a.theta = theta1;
    a.wt = wt1;
    a.lam = lambda;
    a.flag = h->flag;
    a.wscale = 1.0;
    a.kind = KIND_PROBE;
    // interior points, wall points and the normalisation point: the probe layout
    if (h->p.n_pts > 0) {
      JetArgs b = a;
      b.n = h->p.n_pts;
      b.y = h->p.y;
      b.ystride = h->p.n_pts;
      b.r = h->base_int;
      GN_S_TRY(launch_jet(b, st, nullptr));
    }
    if (h->p.n_bnd > 0) {
      JetArgs b = a;
      b.n = h->p.n_bnd;
      b.y = h->p.y_bnd;
      b.ystride = h->p.n_bnd;
      b.r = h->base_wall;
      GN_S_TRY(launch_jet(b, st, nullptr));
    }
    if (h->p.n_inf > 0) {
      JetArgs b = a;
      b.n = h->p.n_inf;
      b.y = h->p.y_inf;
      b.ystride = h->p.n_inf;
      b.r = h->base_inf;
      GN_S_TRY(launch_jet(b, st, nullptr));
    }
    if (h->p.n_relu > 0) {
      JetArgs b = a;
      b.n = h->p.n_relu;
      b.y = h->p.y_relu;
      b.ystride = h->p.n_relu;
      b.r = h->base_relu;
      GN_S_TRY(launch_jet(b, st, nullptr));
    }
    {
      JetArgs b = a;
      b.n = 1;
      b.y = h->red + 512;   // the handle's copy of the normalisation point
      b.ystride = 1;
      b.r = h->base_norm;
      GN_S_TRY(launch_jet(b, st, nullptr));
    }
    // CCF: g_1 at the positive Hilbert nodes
    if (h->eq == GN_CCF) {
      JetArgs b = a;
      b.kind = KIND_NODE;
      b.n = h->Mh;
      b.y = h->snode;
      b.ystride = h->Mh;
      b.r = h->base_node;
      GN_S_TRY(launch_jet(b, st, nullptr));
    }
    GN_S_TRY(cudaStreamSynchronize(st));
    h->staged = 1;
    h->stage_eps = eps;
    h->base_ld = ld;
    h->lam_frozen = 1;
  }
done:
  cudaFree(wt1);
  return rc;
}

}  // extern "C"
