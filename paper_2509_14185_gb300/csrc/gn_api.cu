// Host side of the C ABI (include/gn.h): handle lifecycle, the evaluation
// passes over the point kinds, and the damped Gauss-Newton step driver
// (Methods, "Second-order Optimizer"; constants of the line search and of the
// Levenberg-Marquardt rule are this library's, the paper gives none).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gn_internal.cuh"

using namespace gn;

std::atomic<long long> gn::g_launches{0};

namespace gn {
static thread_local char g_detail[256] = "";
void set_detail(const char* where, int line, const char* what) {
  const char* base = strrchr(where, '/');
  snprintf(g_detail, sizeof(g_detail), "%s:%d: %s", base ? base + 1 : where, line, what);
}
cudaError_t note_cuda(cudaError_t e, const char* where, int line) {
  if (e != cudaSuccess) set_detail(where, line, cudaGetErrorString(e));
  return e;
}
}  // namespace gn

namespace {

#define GN_TRY_CUDA(x)                                      \
  do {                                                      \
    cudaError_t e_ = GN_NOTE(x);                            \
    if (e_ != cudaSuccess) return GN_ERR_CUDA;              \
  } while (0)

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

int dim_of(int eq) { return (eq == GN_IPM || eq == GN_BOUSSINESQ) ? 2 : 1; }
int fields_of(int eq) { return eq == GN_IPM ? 2 : (eq == GN_BOUSSINESQ ? 3 : 1); }
int neq_of(int eq) { return eq == GN_IPM ? 2 : (eq == GN_BOUSSINESQ ? 3 : 1); }

int validate(const gn_problem* p) {
  if (!p) return GN_ERR_INVALID;
  if (p->equation < GN_BURGERS || p->equation > GN_BOUSSINESQ) return GN_ERR_INVALID;
  if (p->n_layers < 1 || p->n_layers > GN_MAX_LAYERS) return GN_ERR_INVALID;
  const int d = dim_of(p->equation);
  if (p->widths[0] != d || p->widths[p->n_layers] != fields_of(p->equation)) return GN_ERR_INVALID;
  for (int l = 1; l < p->n_layers; l++)
    if (p->widths[l] < 1 || p->widths[l] > 256) return GN_ERR_INVALID;
  if (p->n_pts < 0 || (p->n_pts > 0 && !p->y)) return GN_ERR_INVALID;
  if (d == 1 && p->n_bnd != 0) return GN_ERR_INVALID;
  if (p->n_bnd < 0 || (p->n_bnd > 0 && !p->y_bnd)) return GN_ERR_INVALID;
  if (p->n_inf < 0 || (p->n_inf > 0 && !p->y_inf) || !(p->c_inf >= 0.0)) return GN_ERR_INVALID;
  if (p->norm_kind < 0 || p->norm_kind > 2) return GN_ERR_INVALID;
  if (p->output_map < 0 || p->output_map > 1) return GN_ERR_INVALID;
  if (p->row_block < 0) return GN_ERR_INVALID;
  if (p->n_relu < 0 || (p->n_relu > 0 && !p->y_relu) || !(p->c_relu >= 0.0) || !std::isfinite(p->relu_bound))
    return GN_ERR_INVALID;
  if (p->norm_kind > 0 && (p->norm_field < 0 || p->norm_field >= fields_of(p->equation))) return GN_ERR_INVALID;
  if (p->equation == GN_CCF) {
    if (p->hilbert_m < 8 || p->hilbert_m > 16384 || (p->hilbert_m & 1)) return GN_ERR_INVALID;
  }
  if (p->precision < GN_PREC_FP64 || p->precision > GN_PREC_SPLIT_ALL) return GN_ERR_INVALID;
  if (p->fourier_m < 0) return GN_ERR_INVALID;
  if (p->fourier_m > 0 && (p->n_layers < 3 || p->widths[2] != 2 * p->fourier_m || !p->fourier_B))
    return GN_ERR_INVALID;
  if (p->precision != GN_PREC_FP64 && (p->n_slices < 1 || p->n_slices > 6)) return GN_ERR_INVALID;
  if (p->n_d1 < 0 || (p->n_d1 > 0 && !p->y_d1) || !(p->c_d1 >= 0.0)) return GN_ERR_INVALID;
  if (p->n_d2 < 0 || (p->n_d2 > 0 && !p->y_d2) || !(p->c_d2 >= 0.0)) return GN_ERR_INVALID;
  // the derivative rows' kernel covers tanh networks with a linear output layer
  if ((p->n_d1 > 0 || p->n_d2 > 0) && (p->fourier_m > 0 || p->output_map == 1)) return GN_ERR_UNSUPPORTED;
  return GN_OK;
}

int64_t dpow(int d, int k) { return k == 0 ? 1 : (k == 1 ? d : (int64_t)d * d); }

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(T));
}

void free_all(gn_handle* h) {
  void* ptrs[] = {h->ema_ws, h->wt, h->theta_t, h->r, h->J, h->G, h->A, h->Linv, h->g, h->delta, h->vtmp, h->red,
                  h->flag, h->gpart, h->kf, h->dcoef, h->snode, h->gnode, h->Jg, h->ug, h->sU, h->tnode,
                  h->split_ws, h->chol_ws, h->base_int, h->base_wall, h->base_norm, h->base_node, h->fourierW,
                  h->base_inf, h->base_relu, h->kd[0], h->kd[1], h->dd[0], h->dd[1], h->ugd[0], h->ugd[1],
                  h->sUd[0], h->sUd[1]};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->hpin) cudaFreeHost(h->hpin);
}

void destroy_side(gn_handle* h) {
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->st_aux) cudaStreamDestroy(h->st_aux);
  h->ev_fork = h->ev_join = nullptr;
  h->st_aux = nullptr;
}

// Device copy of the normalisation point: red[512 .. 513].
double* norm_point(gn_handle* h) { return h->red + 512; }

// Rows of the derivative-loss batches (ord 1: d1, 2: d2) and the first of each; the wall,
// decay and bound rows follow them.
int64_t n_drows(const gn_handle* h, int ord) {
  return (ord == 1 ? h->p.n_d1 : h->p.n_d2) * h->ne * dpow(h->d, ord);
}
int64_t drow0(const gn_handle* h, int ord) {
  return h->p.n_pts * h->ne + (ord == 2 ? n_drows(h, 1) : 0);
}
int64_t edge_row0(const gn_handle* h) { return h->p.n_pts * h->ne + n_drows(h, 1) + n_drows(h, 2); }

}  // namespace

namespace gn {

// Evaluate rows (all kinds) at (theta, lambda) in one mode.  In gradient mode
// the per-warp partials are reduced into grad (P+1 entries).
int run_pass(gn_handle* h, const double* theta, double lam, const Pass& ps, double* grad) {
  cudaStream_t st = h->st;
  GN_TRY_CUDA(launch_transpose_weights(h->net, theta, h->wt, st));
  JetArgs a;
  memset(&a, 0, sizeof(a));
  a.net = h->net;
  a.eq = h->eq;
  a.theta = theta;
  a.wt = h->wt;
  a.lam = lam;
  a.lamp = ps.lamp;
  a.flag = h->flag;
  a.lam_frozen = h->lam_frozen;
  a.fW = h->fourierW;
  a.eps = h->stage_eps;
  a.base_ld = h->base_ld;
  // the normalisation constraint's field and derivative (the decay rows use the same field)
  a.nfield = h->p.norm_kind > 0 ? h->p.norm_field : 0;
  a.nderiv = h->p.norm_kind == 2 || (h->p.norm_kind == 0 && h->eq == GN_BOUSSINESQ);
  // stage 2: rows are R(Phi_1 + eps Phi_2) / eps (unless the caller wants R itself)
  const double rs = (h->staged && !ps.unweighted) ? 1.0 / h->stage_eps : 1.0;
  a.ldg = round_up(h->Pp, 16);
  a.gpart = h->gpart;
  const int64_t n = h->p.n_pts;
  if (ps.mode == MODE_GRADIENT) GN_TRY_CUDA(cudaMemsetAsync(h->gpart, 0, h->gpart_warps * a.ldg * 8, st));

  // wall points and the normalisation row: rows of their own.  In residual and Jacobian
  // modes they run on the handle's side stream, beside the Hilbert nodes and the interior
  // (a one-point pass is latency-bound; alone it would add its whole latency); gradient mode
  // accumulates every kind into the same per-warp partials, so it keeps them in order.
  const bool side = ps.mode != MODE_GRADIENT && h->st_aux;
  auto edge_rows = [&](cudaStream_t sx) -> int {
    // wall points
    if (h->p.n_bnd > 0) {
      JetArgs b = a;
      b.kind = KIND_WALL;
      b.mode = ps.mode;
      b.n = h->p.n_bnd;
      b.y = h->p.y_bnd;
      b.ystride = h->p.n_bnd;
      b.wscale = rs * sqrt(2.0 * h->p.c_bnd / (double)h->p.n_bnd);
      b.base = h->staged ? h->base_wall : nullptr;
      b.row0 = edge_row0(h);
      b.r = ps.r;
      b.J = ps.J;
      b.ldJ = ps.ldJ;
      b.jrow_lo = ps.jlo;
      b.jrow_hi = ps.jhi;
      b.seed = ps.seed;
      GN_TRY_CUDA(launch_jet(b, sx, nullptr));
    }
    // decay rows of the data loss: sqrt(2 c_inf) Phi_A0 at the far points
    if (h->p.n_inf > 0) {
      JetArgs b = a;
      b.kind = KIND_INF;
      b.mode = ps.mode;
      b.n = h->p.n_inf;
      b.y = h->p.y_inf;
      b.ystride = h->p.n_inf;
      b.wscale = rs * sqrt(2.0 * h->p.c_inf);
      b.base = h->staged ? h->base_inf : nullptr;
      b.c_norm = 0.0;
      b.row0 = edge_row0(h) + h->p.n_bnd;
      b.r = ps.r;
      b.J = ps.J;
      b.ldJ = ps.ldJ;
      b.jrow_lo = ps.jlo;
      b.jrow_hi = ps.jhi;
      b.seed = ps.seed;
      GN_TRY_CUDA(launch_jet(b, sx, nullptr));
    }
    // bound rows of the data loss: sqrt(2 c_relu) relu(s (Phi_A0 - b)) at their points
    if (h->p.n_relu > 0) {
      JetArgs b = a;
      b.kind = KIND_RELU;
      b.mode = ps.mode;
      b.n = h->p.n_relu;
      b.y = h->p.y_relu;
      b.ystride = h->p.n_relu;
      b.wscale = rs * sqrt(2.0 * h->p.c_relu);
      b.base = h->staged ? h->base_relu : nullptr;
      b.c_norm = h->p.relu_bound;
      b.rsign = h->p.relu_sign < 0 ? -1 : 1;
      b.row0 = edge_row0(h) + h->p.n_bnd + h->p.n_inf;
      b.r = ps.r;
      b.J = ps.J;
      b.ldJ = ps.ldJ;
      b.jrow_lo = ps.jlo;
      b.jrow_hi = ps.jhi;
      b.seed = ps.seed;
      GN_TRY_CUDA(launch_jet(b, sx, nullptr));
    }
    // normalisation row
    {
      JetArgs b = a;
      b.kind = KIND_NORM;
      b.mode = ps.mode;
      b.n = 1;
      b.y = norm_point(h);
      b.ystride = 1;
      b.wscale = rs * sqrt(2.0 * h->p.c_norm_w);
      b.base = h->staged ? h->base_norm : nullptr;
      b.c_norm = h->p.c_norm;
      b.row0 = h->n_rows - 1;
      b.r = ps.r;
      b.J = ps.J;
      b.ldJ = ps.ldJ;
      b.jrow_lo = ps.jlo;
      b.jrow_hi = ps.jhi;
      b.seed = ps.seed;
      GN_TRY_CUDA(launch_jet(b, sx, nullptr));
    }
    return GN_OK;
  };
  if (side) {
    GN_TRY_CUDA(cudaEventRecord(h->ev_fork, st));
    GN_TRY_CUDA(cudaStreamWaitEvent(h->st_aux, h->ev_fork, 0));
    int rc = edge_rows(h->st_aux);
    if (rc) return rc;
    GN_TRY_CUDA(cudaEventRecord(h->ev_join, h->st_aux));
  }
  // CCF: g at the positive Hilbert nodes (and their Jacobian rows), then U's K part.
  if (h->eq == GN_CCF) {
    JetArgs b = a;
    b.kind = KIND_NODE;
    b.mode = (ps.mode == MODE_JACOBIAN) ? MODE_JACOBIAN : MODE_RESIDUAL;
    b.n = h->Mh;
    b.y = h->snode;
    b.ystride = h->Mh;
    b.wscale = 1.0;
    b.row0 = 0;
    b.r = h->gnode;
    b.J = h->Jg;
    b.ldJ = h->ldJ;
    b.jrow_lo = 0;
    b.jrow_hi = h->Mh;
    b.base = h->staged ? h->base_node : nullptr;
    b.base_ld = 1;
    GN_TRY_CUDA(launch_jet(b, st, nullptr));
    GN_TRY_CUDA(dgemv_n(h->kf, h->Mh, n, h->Mh, h->gnode, h->ug, 0.0, st));
    // the derivative batches' K part, one coefficient of the series in y at a time
    for (int od = 1; od <= 2; od++) {
      const int64_t nd = od == 1 ? h->p.n_d1 : h->p.n_d2;
      for (int m = 0; nd > 0 && m <= djet_order_y(1, od); m++)
        GN_TRY_CUDA(dgemv_n(h->kd[od - 1] + (int64_t)m * nd * h->Mh, h->Mh, nd, h->Mh, h->gnode,
                            h->ugd[od - 1] + (int64_t)m * nd, 0.0, st));
    }
  }
  // interior points
  {
    JetArgs b = a;
    b.kind = KIND_INTERIOR;
    b.mode = ps.mode;
    b.n = n;
    b.y = h->p.y;
    b.ystride = n;
    b.rho = ps.unweighted ? nullptr : h->p.rho;
    b.wscale = ps.unweighted ? 1.0 : rs * (n > 0 ? sqrt(2.0 / ((double)n * h->ne)) : 0.0);
    b.base = h->staged ? h->base_int : nullptr;
    b.row0 = 0;
    b.r = ps.r;
    b.J = ps.J;
    b.ldJ = ps.ldJ;
    b.jrow_lo = ps.jlo;
    b.jrow_hi = ps.jhi;
    b.seed = ps.seed;
    b.ug = h->ug;
    b.dcoef = h->dcoef;
    b.sU = h->sU;
    GN_TRY_CUDA(launch_jet(b, st, nullptr));
  }
  // derivative-loss rows (d1, d2)
  for (int od = 1; od <= 2; od++) {
    const int64_t nd = od == 1 ? h->p.n_d1 : h->p.n_d2;
    if (nd == 0) continue;
    JetArgs b = a;
    b.mode = ps.mode;
    b.n = nd;
    b.y = od == 1 ? h->p.y_d1 : h->p.y_d2;
    b.ystride = nd;
    b.rho = ps.unweighted ? nullptr : (od == 1 ? h->p.rho_d1 : h->p.rho_d2);
    const double cd = od == 1 ? h->p.c_d1 : h->p.c_d2;
    b.wscale = ps.unweighted ? 1.0 : rs * sqrt(2.0 * cd / ((double)nd * h->ne * dpow(h->d, od)));
    b.base = nullptr;
    b.row0 = drow0(h, od);
    b.r = ps.r;
    b.J = ps.J;
    b.ldJ = ps.ldJ;
    b.jrow_lo = ps.jlo;
    b.jrow_hi = ps.jhi;
    b.seed = ps.seed;
    b.ug = h->ugd[od - 1];
    b.dcoef = h->dd[od - 1];
    b.sU = h->sUd[od - 1];
    GN_TRY_CUDA(launch_djet(b, od, st, nullptr));
    if (h->eq == GN_CCF && ps.mode == MODE_JACOBIAN) {
      // J[row, :] += sum_m sU_m(row) sum_j' Kd_m[row][j'] Jg[j', :] (one row per point in 1D)
      const int64_t r0 = b.row0;
      const int64_t lo = ps.jlo > r0 ? ps.jlo : r0, hi = ps.jhi < r0 + nd ? ps.jhi : r0 + nd;
      for (int m = 0; hi > lo && m <= od; m++)
        GN_TRY_CUDA(dgemm(hi - lo, h->Pp, h->Mh, 1.0, h->kd[od - 1] + ((int64_t)m * nd + (lo - r0)) * h->Mh, h->Mh,
                          true, h->Jg, h->ldJ, false, 1.0, ps.J + (lo - ps.jlo) * ps.ldJ, ps.ldJ, false,
                          h->sUd[od - 1] + (int64_t)m * nd + (lo - r0), st));
    }
  }
  if (!side) {
    int rc = edge_rows(st);
    if (rc) return rc;
  }
  if (h->eq == GN_CCF && ps.mode == MODE_JACOBIAN) {
    // J[i, :] += sU_i * sum_j' Kf[i][j'] Jg[j', :] for interior rows inside the block
    const int64_t lo = ps.jlo > 0 ? ps.jlo : 0;
    const int64_t hi = ps.jhi < n ? ps.jhi : n;
    if (hi > lo && h->precision == GN_PREC_SPLIT_ALL) {
      // the same contraction as a split GEMM on the tensor cores: A = Kf rows
      // (row-scaled), B = J_g columns (column-scaled), C += sU_i * value
      const int S = h->n_slices;
      const size_t ba = oz_operand_bytes(S, hi - lo, h->Mh), bb = oz_operand_bytes(S, h->Pp, h->Mh);
      const size_t bp = (size_t)64 * ((h->Pp + 127) / 128 * 128) * 8;
      int rc = ensure_split_ws(h, ba + bb + bp + 512);
      if (rc) return rc;
      unsigned char* base = static_cast<unsigned char*>(h->split_ws);
      OzOperand A = oz_operand_at(base, S, hi - lo, h->Mh);
      OzOperand B = oz_operand_at(base + ba, S, h->Pp, h->Mh);
      double* part = reinterpret_cast<double*>(base + ba + bb);
      rc = oz_prepare_rows(S, h->kf + lo * h->Mh, h->Mh, hi - lo, h->Mh, A, st);
      if (!rc) rc = oz_prepare_cols(S, h->Jg, h->ldJ, h->Mh, h->Pp, B, part, st);
      if (!rc)
        rc = oz_gemm(S, false, A, B, hi - lo, h->Pp, ps.J + (lo - ps.jlo) * ps.ldJ, ps.ldJ, 1, h->sU + lo,
                     h->flag + 2, st);
      if (rc) return rc;
    } else if (hi > lo) {
      GN_TRY_CUDA(dgemm(hi - lo, h->Pp, h->Mh, 1.0, h->kf + lo * h->Mh, h->Mh, true, h->Jg, h->ldJ, false, 1.0,
                        ps.J + (lo - ps.jlo) * ps.ldJ, ps.ldJ, false, h->sU + lo, st));
    }
  }
  if (side) GN_TRY_CUDA(cudaStreamWaitEvent(st, h->ev_join, 0));
  if (ps.mode == MODE_GRADIENT) {
    if (h->eq == GN_CCF && n > 0) {
      // t_j' = sum_i Kf[i][j'] c_i (c = seed * w * dR/dU, left in sU), then node pass seeded by t
      GN_TRY_CUDA(dgemv_t_scratch(h->kf, h->Mh, n, h->Mh, h->sU, h->tnode, 0.0, h->vtmp, st));
      for (int od = 1; od <= 2; od++) {   // the derivative rows' K parts, coefficient by coefficient
        const int64_t nd = od == 1 ? h->p.n_d1 : h->p.n_d2;
        for (int m = 0; nd > 0 && m <= od; m++)
          GN_TRY_CUDA(dgemv_t_scratch(h->kd[od - 1] + (int64_t)m * nd * h->Mh, h->Mh, nd, h->Mh,
                                      h->sUd[od - 1] + (int64_t)m * nd, h->tnode, 1.0, h->vtmp, st));
      }
      JetArgs b = a;
      b.kind = KIND_NODE;
      b.mode = MODE_GRADIENT;
      b.n = h->Mh;
      b.y = h->snode;
      b.ystride = h->Mh;
      b.wscale = 1.0;
      b.row0 = 0;
      b.r = nullptr;
      b.seed = h->tnode;
      b.base = h->staged ? h->base_node : nullptr;
      b.base_ld = 1;
      GN_TRY_CUDA(launch_jet(b, st, nullptr));
    }
    GN_TRY_CUDA(launch_gpart_reduce(h->gpart, h->gpart_warps, a.ldg, h->Pp, grad, 0, st));
  }
  return GN_OK;
}

// loss = 1/2 |r|^2 into hpin[slot] (device copy, then host after sync)
int loss_of(gn_handle* h, const double* r, int slot) {
  GN_TRY_CUDA(sumsq_and_flag(r, h->n_rows, h->red, h->st));
  GN_TRY_CUDA(finish_sum(h->red, h->red + 256 + slot, h->st));
  return GN_OK;
}

int max_res_of(gn_handle* h, const double* r) {
  const int64_t n = h->p.n_pts;
  if (n == 0) {
    GN_TRY_CUDA(cudaMemsetAsync(h->red + kMaxResSlot, 0, sizeof(double), h->st));
    return GN_OK;
  }
  // interior rows carry sqrt(2 rho / (N N_E)) R_k, divided by eps in a second stage
  const double w = sqrt(2.0 / ((double)n * h->ne)) / (h->staged ? h->stage_eps : 1.0);
  GN_TRY_CUDA(max_abs_unweighted(r, n, h->ne, h->p.rho, w, h->red, h->red + kMaxResSlot, h->st));
  return GN_OK;
}

int residual_loss(gn_handle* h, const double* theta, double lam, double* r, double* loss) {
  Pass ps = {MODE_RESIDUAL, r, nullptr, 0, 0, 0, nullptr};
  int rc = run_pass(h, theta, lam, ps, nullptr);
  if (rc) return rc;
  if (loss) {
    rc = loss_of(h, r, 0);
    if (rc) return rc;
    GN_TRY_CUDA(cudaMemcpyAsync(h->hpin, h->red + 256, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    GN_TRY_CUDA(cudaStreamSynchronize(h->st));
    *loss = 0.5 * h->hpin[0];
  }
  return GN_OK;
}

int gram_into(gn_handle* h, const double* J, int64_t ld, int64_t nrows, const double* r, double* G, double* g,
              int precision, int accumulate) {
  const double beta = accumulate ? 1.0 : 0.0;
  if (precision != GN_PREC_FP64) {
    int rc = split_gram(h, J, ld, nrows, G, accumulate);
    if (rc) return rc;
  } else {
    GN_TRY_CUDA(dgemm(h->Pp, h->Pp, nrows, 1.0, J, ld, false, J, ld, false, beta, G, h->Pp, true, nullptr, h->st));
  }
  if (r && g) GN_TRY_CUDA(dgemv_t_scratch(J, ld, nrows, h->Pp, r, g, beta, h->vtmp, h->st));
  return GN_OK;
}

}  // namespace gn

namespace {

// NVTX ranges naming the host-side phases of a step (shown by Nsight Systems; no-ops when no
// tool is attached).
struct Phases {
  bool open = false;
  void next(const char* name) {
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~Phases() {
    if (open) nvtxRangePop();
  }
};

struct Timer {
  cudaEvent_t ev[9];
  int n = 0;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    for (auto& e : ev) cudaEventCreate(&e);
  }
  ~Timer() {
    for (auto& e : ev) cudaEventDestroy(e);
  }
  void mark(int i) { cudaEventRecord(ev[i], st); }
  double ms(int a, int b) {
    float v = 0.f;
    cudaEventElapsedTime(&v, ev[a], ev[b]);
    return v;
  }
};

}  // namespace

extern "C" {

const char* gn_last_error_detail(void) { return g_detail; }

int64_t gn_kernel_launches(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

const char* gn_error_string(int code) {
  switch (code) {
    case GN_OK: return "ok";
    case GN_WARN_NO_DECREASE: return "line search found no decrease; step rejected, damping raised";
    case GN_ERR_INVALID: return "invalid argument";
    case GN_ERR_CUDA: return "CUDA runtime error";
    case GN_ERR_OOM: return "device allocation failed";
    case GN_ERR_NONFINITE: return "non-finite residual or loss";
    case GN_ERR_NOT_SPD: return "damped Gauss-Newton matrix not positive definite";
    case GN_ERR_TIMEOUT: return "bounded device wait timed out";
    case GN_ERR_UNSUPPORTED: return "unsupported on this device or build";
    case GN_ERR_TOO_LARGE: return "size exceeds the fixed scratch of the allocation-free entry point";
    case GN_ERR_IO: return "checkpoint file could not be written or read";
    case GN_ERR_MISMATCH: return "checkpoint belongs to another equation or architecture";
    default: return "unknown status";
  }
}

int gn_init(const gn_problem* p, void* cuda_stream, gn_handle** out) {
  if (!out) return GN_ERR_INVALID;
  *out = nullptr;
  int rc = validate(p);
  if (rc) return rc;
  gn_handle* h = new (std::nothrow) gn_handle;
  if (!h) return GN_ERR_OOM;
  memset(h, 0, sizeof(*h));
  h->p = *p;
  if (h->p.n_pts == 0) h->p.y = nullptr;
  GN_TRY_CUDA(cudaGetDevice(&h->dev));
  h->st = (cudaStream_t)cuda_stream;
  h->eq = p->equation;
  h->d = dim_of(h->eq);
  h->nf = fields_of(h->eq);
  h->ne = neq_of(h->eq);
  NetDesc& net = h->net;
  net.L = p->n_layers;
  net.maxw = 2;
  int64_t off = 0, offT = 0;
  for (int l = 0; l <= net.L; l++) {
    net.w[l] = p->widths[l];
    if (net.w[l] > net.maxw) net.maxw = net.w[l];
  }
  net.fourier = p->fourier_m > 0 ? 1 : 0;
  net.exp_out = p->output_map == 1 ? 1 : 0;
  for (int l = 0; l < net.L; l++) {
    net.offT[l] = offT;
    offT += (int64_t)net.w[l] * net.w[l + 1];
    if (net.fourier && l == 1) {   // the fixed Fourier map takes no place in theta
      net.offW[l] = -1;
      net.offB[l] = -1;
      continue;
    }
    net.offW[l] = off;
    off += (int64_t)net.w[l] * net.w[l + 1];
    net.offB[l] = off;
    off += net.w[l + 1];
  }
  net.P = off;
  h->P = off;
  h->Pp = off + 1;
  h->n_rows = p->n_pts * h->ne + p->n_d1 * h->ne * dpow(h->d, 1) + p->n_d2 * h->ne * dpow(h->d, 2) +
              (h->d == 2 ? p->n_bnd : 0) + p->n_inf + p->n_relu + 1;
  h->ldJ = round_up(h->Pp, 16);
  const double jbytes = (double)h->n_rows * h->ldJ * 8.0;
  const double jcap = 32.0 * (1ull << 30);
  h->jrows = jbytes <= jcap ? h->n_rows : (int64_t)(jcap / (h->ldJ * 8.0));
  if (p->row_block > 0 && p->row_block < h->jrows) h->jrows = p->row_block;   // the caller's block
  h->precision = p->precision;
  h->n_slices = p->n_slices > 0 ? p->n_slices : 4;
  h->gpart_warps = jet_gpart_warps(net, h->d, h->nf, p->n_pts);

  bool ok = true;
  auto A = [&](cudaError_t e) {
    if (e != cudaSuccess) ok = false;
  };
  const int64_t Pp = h->Pp;
  const int64_t nvec = (Pp > h->n_rows ? Pp : h->n_rows);
  A(dalloc(&h->wt, offT > h->P ? offT : h->P));
  if (net.fourier) A(dalloc(&h->fourierW, (size_t)net.w[2] * net.w[1]));
  A(dalloc(&h->theta_t, h->P));
  A(dalloc(&h->r, h->n_rows));
  if (ok) A(dalloc(&h->J, (size_t)h->jrows * h->ldJ));
  if (ok) A(dalloc(&h->G, (size_t)Pp * Pp));
  if (ok) A(dalloc(&h->A, (size_t)Pp * Pp));
  A(dalloc(&h->Linv, (size_t)((Pp + kCholNB - 1) / kCholNB) * kCholNB * kCholNB));
  A(dalloc(&h->g, Pp));
  A(dalloc(&h->delta, Pp));
  A(dalloc(&h->vtmp, (size_t)kGemvChunks * (nvec + 16)));
  A(dalloc(&h->red, 1024));
  A(dalloc(&h->flag, 4));
  if (ok) A(dalloc(&h->gpart, (size_t)h->gpart_warps * round_up(Pp, 16)));
  if (cudaMallocHost((void**)&h->hpin, 64 * sizeof(double)) != cudaSuccess) ok = false;
  if (h->eq == GN_CCF) {
    h->M = p->hilbert_m;
    h->Mh = h->M / 2;
    A(dalloc(&h->kf, (size_t)p->n_pts * h->Mh));
    A(dalloc(&h->dcoef, p->n_pts));
    A(dalloc(&h->snode, h->Mh));
    A(dalloc(&h->gnode, h->Mh));
    A(dalloc(&h->Jg, (size_t)h->Mh * h->ldJ));
    A(dalloc(&h->ug, p->n_pts));
    A(dalloc(&h->sU, p->n_pts));
    A(dalloc(&h->tnode, h->Mh));
    for (int od = 1; od <= 2; od++) {
      const int64_t nd = od == 1 ? p->n_d1 : p->n_d2;
      if (nd == 0) continue;
      const int oy = djet_order_y(1, od);
      A(dalloc(&h->kd[od - 1], (size_t)(oy + 1) * nd * h->Mh));
      A(dalloc(&h->dd[od - 1], (size_t)(oy + 1) * nd));
      A(dalloc(&h->ugd[od - 1], (size_t)(oy + 1) * nd));
      A(dalloc(&h->sUd[od - 1], (size_t)(od + 1) * nd));
    }
  }
  if (!ok) {
    cudaGetLastError();
    free_all(h);
    delete h;
    return GN_ERR_OOM;
  }
  cudaError_t e = cudaMemsetAsync(h->flag, 0, 4 * sizeof(int), h->st);
  if (e == cudaSuccess && net.fourier) {
    // rows [B; B] (cos half, sin half) and their transposed copy at offT[1] of the weight copy
    const int m = net.w[1], mf = net.w[2] / 2;
    std::vector<double> rows((size_t)2 * mf * m), tr((size_t)2 * mf * m);
    for (int o = 0; o < 2 * mf; o++)
      for (int i = 0; i < m; i++) rows[(size_t)o * m + i] = p->fourier_B[(size_t)(o % mf) * m + i];
    for (int i = 0; i < m; i++)
      for (int o = 0; o < 2 * mf; o++) tr[(size_t)i * 2 * mf + o] = rows[(size_t)o * m + i];
    e = cudaMemcpy(h->fourierW, rows.data(), rows.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(h->wt + net.offT[1], tr.data(), tr.size() * sizeof(double), cudaMemcpyHostToDevice);
  }
  double yn[2] = {p->y_norm[0], p->y_norm[1]};
  if (e == cudaSuccess) e = cudaMemcpyAsync(norm_point(h), yn, 2 * sizeof(double), cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess && h->eq == GN_CCF) e = hilbert_build(p->y, p->n_pts, h->M, h->kf, h->dcoef, h->snode, h->st);
  for (int od = 1; od <= 2 && e == cudaSuccess && h->eq == GN_CCF; od++) {
    const int64_t nd = od == 1 ? p->n_d1 : p->n_d2;
    if (nd > 0)
      e = hilbert_series_build(od == 1 ? p->y_d1 : p->y_d2, nd, h->M, djet_order_y(1, od), h->kd[od - 1],
                               h->dd[od - 1], h->st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  // the side stream of the wall and normalisation passes (highest priority: a one-CTA pass
  // should not queue behind the interior pass's CTAs)
  if (e == cudaSuccess) {
    int least = 0, greatest = 0;
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->st_aux, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    destroy_side(h);
    free_all(h);
    delete h;
    return GN_ERR_CUDA;
  }
  *out = h;
  return GN_OK;
}

int gn_destroy(gn_handle* h) {
  if (!h) return GN_OK;
  cudaStreamSynchronize(h->st);
  graph_release(h);
  if (h->st_hi) cudaStreamDestroy(h->st_hi);
  if (h->st_lo) cudaStreamDestroy(h->st_lo);
  if (h->st_g) cudaStreamDestroy(h->st_g);
  destroy_side(h);
  free_all(h);
  if (h->tmaps) free(h->tmaps);
  delete h;
  return GN_OK;
}

int gn_param_count(const gn_handle* h, int64_t* P) {
  if (!h || !P) return GN_ERR_INVALID;
  *P = h->P;
  return GN_OK;
}

int gn_row_count(const gn_handle* h, int64_t* n_rows) {
  if (!h || !n_rows) return GN_ERR_INVALID;
  *n_rows = h->n_rows;
  return GN_OK;
}

int gn_set_precision(gn_handle* h, int precision, int n_slices) {
  if (!h) return GN_ERR_INVALID;
  if (precision < GN_PREC_FP64 || precision > GN_PREC_SPLIT_ALL) return GN_ERR_INVALID;
  if (precision != GN_PREC_FP64 && (n_slices < 1 || n_slices > 6)) return GN_ERR_INVALID;
  h->precision = precision;
  if (n_slices > 0) h->n_slices = n_slices;
  return GN_OK;
}

int gn_set_gram_split(gn_handle* h, int ksplit) {
  if (!h || ksplit < 0 || ksplit > 8) return GN_ERR_INVALID;
  h->gram_ksplit = ksplit;
  return GN_OK;
}

int gn_set_pipeline(gn_handle* h, int tiles) {
  if (!h || tiles < -1) return GN_ERR_INVALID;
  h->pipe_tiles = tiles;
  return GN_OK;
}

int gn_pipeline_tiles(gn_handle* h, int64_t* tiles) {
  if (!h || !tiles) return GN_ERR_INVALID;
  *tiles = pipeline_chunk_tiles(h);
  return GN_OK;
}

int gn_set_gram_tile(gn_handle* h, int tile_n) {
  if (!h || (tile_n != 0 && tile_n != 64 && tile_n != 128)) return GN_ERR_INVALID;
  h->gram_tile = tile_n;
  return GN_OK;
}

int gn_gram_tile_choice(const gn_handle* h, int64_t nrows, int* tile_n) {
  if (!h || !tile_n || nrows < 0) return GN_ERR_INVALID;
  *tile_n = h->gram_tile > 0 ? h->gram_tile : gram_tile_choice(h->n_slices, h->Pp, nrows);
  return GN_OK;
}

int gn_gram_split_choice(const gn_handle* h, int64_t nrows, int* ksplit) {
  if (!h || !ksplit || nrows < 0) return GN_ERR_INVALID;
  *ksplit = h->gram_ksplit > 0 ? h->gram_ksplit : gram_split_choice(h->n_slices, h->Pp, nrows);
  return GN_OK;
}

int gn_residual(gn_handle* h, const double* theta, double lambda, double* r_out, double* loss_out) {
  if (!h || !theta) return GN_ERR_INVALID;
  double* r = r_out ? r_out : h->r;
  double loss = 0.0;
  int rc = residual_loss(h, theta, lambda, r, loss_out ? &loss : nullptr);
  if (rc) return rc;
  if (loss_out) {
    *loss_out = loss;
    if (!std::isfinite(loss)) return GN_ERR_NONFINITE;
  }
  return GN_OK;
}

int gn_jacobian(gn_handle* h, const double* theta, double lambda, double* J_out, int64_t ld, int64_t row0,
                int64_t nrows) {
  if (!h || !theta || !J_out || ld < h->Pp || row0 < 0 || nrows < 0 || row0 + nrows > h->n_rows)
    return GN_ERR_INVALID;
  if (nrows == 0) return GN_OK;
  Pass ps = {MODE_JACOBIAN, h->r, J_out, ld, row0, row0 + nrows, nullptr};
  return run_pass(h, theta, lambda, ps, nullptr);
}

int gn_gradient(gn_handle* h, const double* theta, double lambda, const double* seed, double* grad_out) {
  if (!h || !theta || !grad_out) return GN_ERR_INVALID;
  Pass ps = {MODE_GRADIENT, h->r, nullptr, 0, 0, 0, seed};
  return run_pass(h, theta, lambda, ps, grad_out);
}

int gn_gram(gn_handle* h, const double* J, int64_t ld, int64_t nrows, const double* r, double* G_out, double* g_out,
            int precision, int accumulate) {
  if (!h || !J || !G_out || ld < h->Pp || nrows < 0) return GN_ERR_INVALID;
  if (precision < GN_PREC_FP64 || precision > GN_PREC_SPLIT_ALL) return GN_ERR_INVALID;
  if (precision == GN_PREC_FP64) return gram_into(h, J, ld, nrows, r, G_out, g_out, precision, accumulate);
  // split precision: report a timed-out tensor-core wait before returning
  GN_TRY_CUDA(cudaMemsetAsync(h->flag + 2, 0, sizeof(int), h->st));
  int rc = gram_into(h, J, ld, nrows, r, G_out, g_out, precision, accumulate);
  if (rc) return rc;
  GN_TRY_CUDA(cudaMemcpyAsync(&h->hpin[9], h->flag + 2, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  GN_TRY_CUDA(cudaStreamSynchronize(h->st));
  int f = 0;
  memcpy(&f, &h->hpin[9], sizeof(int));
  return (f & 2) ? GN_ERR_TIMEOUT : GN_OK;
}

namespace {
// The damped solve of gn_damped_solve.  With check_rows, a non-finite residual row seen by the
// jet kernel since the caller cleared status bit 0 (h->flag[0]) ends the call with
// GN_ERR_NONFINITE at the first synchronisation, before any damping escalation.
int damped_solve(gn_handle* h, const double* G, const double* g, double* gamma, double* delta_out,
                 int* retries_out, bool check_rows) {
  const int64_t Pp = h->Pp;
  int retries = 0;
  for (;;) {
    GN_TRY_CUDA(copy_add_diag(G, h->A, Pp, Pp, *gamma, nullptr, h->st));
    GN_TRY_CUDA(cudaMemsetAsync(h->flag + 1, 0, sizeof(int), h->st));
    if (h->precision == GN_PREC_SPLIT_ALL) {
      int rc = GN_OK;
      cudaError_t e = cholesky_factor_split(h, h->A, Pp, Pp, h->Linv, h->flag + 1, h->n_slices, g, h->vtmp + Pp,
                                            h->vtmp, &rc);
      if (rc) return rc;
      GN_TRY_CUDA(e);
    } else {
      GN_TRY_CUDA(cholesky_factor(h->A, Pp, Pp, h->Linv, h->flag + 1, h->st));
    }
    int hflag[3] = {0, 0, 0};
    GN_TRY_CUDA(cudaMemcpyAsync(&h->hpin[8], h->flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, h->st));
    GN_TRY_CUDA(cudaStreamSynchronize(h->st));
    memcpy(hflag, &h->hpin[8], 3 * sizeof(int));
    if (hflag[2] & 2) {
      set_detail(__FILE__, __LINE__, "a bounded wait in a tensor-core kernel timed out");
      return GN_ERR_TIMEOUT;
    }
    if (check_rows && (hflag[0] & 1)) return GN_ERR_NONFINITE;
    if (!hflag[1]) break;
    if (retries == 5) {
      if (retries_out) *retries_out = retries;
      return GN_ERR_NOT_SPD;
    }
    *gamma *= 10.0;
    retries++;
  }
  if (retries_out) *retries_out = retries;
  // vtmp holds >= 2 Pp doubles: the work vector and (split path) the forward result y
  if (h->precision == GN_PREC_SPLIT_ALL)
    GN_TRY_CUDA(cholesky_solve_backward(h->A, Pp, Pp, h->Linv, h->vtmp + Pp, delta_out, h->vtmp, h->st));
  else
    GN_TRY_CUDA(cholesky_solve(h->A, Pp, Pp, h->Linv, g, delta_out, h->vtmp, h->st));
  return GN_OK;
}
}  // namespace

int gn_damped_solve(gn_handle* h, const double* G, const double* g, double* gamma, double* delta_out,
                    int* retries_out) {
  if (!h || !G || !g || !gamma || !delta_out) return GN_ERR_INVALID;
  return damped_solve(h, G, g, gamma, delta_out, retries_out, false);
}

int gn_max_residual(gn_handle* h, const double* theta, double lambda, double* out) {
  if (!h || !theta || !out) return GN_ERR_INVALID;
  // unweighted interior residuals: evaluate with unit row weights into r
  Pass ps = {MODE_RESIDUAL, h->r, nullptr, 0, 0, 0, nullptr};
  int rc = run_pass(h, theta, lambda, ps, nullptr);
  if (rc) return rc;
  const int64_t nint = h->p.n_pts * h->ne;
  // rows carry sqrt(2 rho/(N N_E)); undo it for rho == 1 (documented: max over unweighted R_k)
  GN_TRY_CUDA(max_abs_rows(h->r, nint, 0, h->red, h->st));
  GN_TRY_CUDA(finish_max(h->red, h->red + 300, h->st));
  GN_TRY_CUDA(cudaMemcpyAsync(h->hpin, h->red + 300, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  GN_TRY_CUDA(cudaStreamSynchronize(h->st));
  const double w = nint > 0 ? sqrt(2.0 / ((double)h->p.n_pts * h->ne)) : 1.0;
  *out = h->hpin[0] / w * (h->staged ? h->stage_eps : 1.0);   // stage 2: max |R| of Phi_1 + eps Phi_2
  return GN_OK;
}

int gn_step(gn_handle* h, double* theta, double* lambda, double* damping, gn_step_info* info) {
  if (!h || !theta || !lambda || !damping) return GN_ERR_INVALID;
  gn_step_info inf;
  memset(&inf, 0, sizeof(inf));
  cudaStream_t st = h->st;
  const int64_t Pp = h->Pp, P = h->P;
  const double lam = *lambda;
  double gamma = *damping;
  Timer tm(st);
  Phases ph;
  // status bits: [0] non-finite residual rows of this step's passes, [2] a timed-out wait
  GN_TRY_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), st));
  GN_TRY_CUDA(cudaMemsetAsync(h->flag + 2, 0, sizeof(int), st));
  tm.mark(0);
  // 1. rows and Jacobian, Gram and gradient, streamed in row blocks
  int rc = GN_OK;
  const int64_t nblk = (h->n_rows + h->jrows - 1) / h->jrows;
  double t_jac = 0.0, t_gram = 0.0;
  for (int64_t b = 0; b < nblk; b++) {
    const int64_t lo = b * h->jrows;
    const int64_t hi = (lo + h->jrows < h->n_rows) ? lo + h->jrows : h->n_rows;
    Pass ps = {MODE_JACOBIAN, h->r, h->J, h->ldJ, lo, hi, nullptr};
    tm.mark(1);
    ph.next("gn_step: jacobian");
    rc = run_pass(h, theta, lam, ps, nullptr);
    if (rc) return rc;
    tm.mark(2);
    ph.next("gn_step: gram");
    rc = gram_into(h, h->J, h->ldJ, hi - lo, h->r + lo, h->G, h->g, h->precision, b > 0);
    if (rc) return rc;
    tm.mark(3);
    if (nblk > 1) {
      GN_TRY_CUDA(cudaEventSynchronize(tm.ev[3]));
      t_jac += tm.ms(1, 2);
      t_gram += tm.ms(2, 3);
    }
  }
  rc = loss_of(h, h->r, 0);
  if (!rc) rc = max_res_of(h, h->r);
  if (rc) return rc;
  GN_TRY_CUDA(cudaMemcpyAsync(h->hpin + 4, h->red + kMaxResSlot, sizeof(double), cudaMemcpyDeviceToHost, st));
  tm.mark(4);
  if (nblk == 1) {
    GN_TRY_CUDA(cudaEventSynchronize(tm.ev[4]));
    t_jac = tm.ms(1, 2);
    t_gram = tm.ms(2, 3);
  }
  // 2. damped solve
  ph.next("gn_step: damped solve");
  int retries = 0;
  rc = damped_solve(h, h->G, h->g, &gamma, h->delta, &retries, true);
  tm.mark(5);
  inf.chol_retries = retries;
  inf.gamma_used = gamma;
  if (rc) {
    inf.status = rc;
    if (info) *info = inf;
    return rc;
  }
  // 3. scalars for the model: g.delta, delta.G.delta, delta[P], h0
  GN_TRY_CUDA(dot_partial(h->g, h->delta, Pp, h->red, st));
  GN_TRY_CUDA(finish_sum(h->red, h->red + 257, st));
  // delta.G.delta from G's lower triangle (the step never forms the upper one)
  GN_TRY_CUDA(quad_lower(h->G, Pp, Pp, h->delta, h->vtmp, st));
  GN_TRY_CUDA(dot_partial(h->delta, h->vtmp, Pp, h->red, st));
  GN_TRY_CUDA(finish_sum(h->red, h->red + 258, st));
  GN_TRY_CUDA(cudaMemcpyAsync(h->red + 259, h->delta + P, sizeof(double), cudaMemcpyDeviceToDevice, st));
  GN_TRY_CUDA(cudaMemcpyAsync(h->hpin, h->red + 256, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  GN_TRY_CUDA(cudaStreamSynchronize(st));
  const double h0 = 0.5 * h->hpin[0];
  const double gd = h->hpin[1];
  const double dGd = h->hpin[2];
  const double dlam = h->hpin[3];
  inf.loss_before = h0;
  inf.loss_after = h0;
  inf.max_abs_res = h->hpin[4];
  tm.mark(6);
  if (!std::isfinite(h0)) {
    inf.status = GN_ERR_NONFINITE;
    if (info) *info = inf;
    return GN_ERR_NONFINITE;
  }
  // 4. Armijo backtracking on residual-only evaluations
  ph.next("gn_step: line search");
  const double c1 = 1e-4;
  double alpha = 1.0;
  bool accepted = false;
  double ht = h0;
  for (int trial = 0; trial < 8; trial++) {
    GN_TRY_CUDA(axpy_trial(theta, h->delta, alpha, P, h->theta_t, st));
    const double lt = lam - alpha * dlam;
    rc = residual_loss(h, h->theta_t, lt, h->r, &ht);
    if (rc) return rc;
    inf.n_trials = trial + 1;
    if (std::isfinite(ht) && ht <= h0 - c1 * alpha * gd) {
      accepted = true;
      break;
    }
    alpha *= 0.5;
  }
  tm.mark(7);
  if (accepted) {
    const double pred = alpha * gd - 0.5 * alpha * alpha * dGd;
    const double rho = pred != 0.0 ? (h0 - ht) / pred : 1.0;
    if (rho < 0.25) gamma *= 1.5;
    else if (rho > 0.75) gamma *= 2.0 / 3.0;
    GN_TRY_CUDA(cudaMemcpyAsync(theta, h->theta_t, P * sizeof(double), cudaMemcpyDeviceToDevice, st));
    *lambda = lam - alpha * dlam;
    inf.alpha = alpha;
    inf.rho = rho;
    inf.loss_after = ht;
    inf.status = GN_OK;
  } else {
    gamma *= 10.0;
    inf.status = GN_WARN_NO_DECREASE;
  }
  *damping = gamma;
  tm.mark(8);
  GN_TRY_CUDA(cudaEventSynchronize(tm.ev[8]));
  inf.ms_phase[0] = t_jac;
  inf.ms_phase[1] = t_gram;
  inf.ms_phase[2] = 0.0;
  inf.ms_phase[3] = tm.ms(4, 5);
  inf.ms_phase[4] = tm.ms(5, 6);
  inf.ms_phase[5] = tm.ms(6, 7);
  inf.ms_phase[6] = tm.ms(0, 8);
  if (info) *info = inf;
  return inf.status;
}

// The paper's own optimiser: EMA of rank-1 curvature estimates, closed-form learning rate
// and momentum (Methods, "Second-order Optimizer"; the readings are listed with the
// declaration in gn.h).
int gn_step_ema(gn_handle* h, double* theta, double* lambda, double* damping, double* G_ema, double* v_prev,
                const double* signs, double beta, int first, gn_step_info* info) {
  if (!h || !theta || !lambda || !damping || !G_ema || !v_prev || !signs || !(beta >= 0.0 && beta < 1.0))
    return GN_ERR_INVALID;
  if (h->jrows < h->n_rows) {
    set_detail(__FILE__, __LINE__, "gn_step_ema needs the whole Jacobian in one block");
    return GN_ERR_UNSUPPORTED;
  }
  gn_step_info inf;
  memset(&inf, 0, sizeof(inf));
  cudaStream_t st = h->st;
  const int64_t Pp = h->Pp, P = h->P, R = h->n_rows;
  const double lam = *lambda;
  double gamma = *damping;
  if (h->ema_len < Pp + 2 * R) {
    if (h->ema_ws) cudaFree(h->ema_ws);
    h->ema_ws = nullptr;
    h->ema_len = 0;
    if (GN_NOTE(dalloc(&h->ema_ws, (size_t)(Pp + 2 * R))) != cudaSuccess) return GN_ERR_OOM;
    h->ema_len = Pp + 2 * R;
  }
  double* u = h->ema_ws;
  double* JD = u + Pp;   // J~ delta
  double* Jv = JD + R;   // J~ v_prev
  Timer tm(st);
  GN_TRY_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), st));
  GN_TRY_CUDA(cudaMemsetAsync(h->flag + 2, 0, sizeof(int), st));
  tm.mark(0);
  // 1. rows and the Jacobian
  Pass ps = {MODE_JACOBIAN, h->r, h->J, h->ldJ, 0, R, nullptr};
  int rc = run_pass(h, theta, lam, ps, nullptr);
  if (rc) return rc;
  tm.mark(1);
  // 2. g = J~^T r~, the rank-1 sample u = J~^T v, its average, h0
  GN_TRY_CUDA(dgemv_t_scratch(h->J, h->ldJ, R, Pp, h->r, h->g, 0.0, h->vtmp, st));
  GN_TRY_CUDA(dgemv_t_scratch(h->J, h->ldJ, R, Pp, signs, u, 0.0, h->vtmp, st));
  rc = loss_of(h, h->r, 0);
  if (rc) return rc;
  GN_TRY_CUDA(ema_rank1(G_ema, Pp, Pp, u, beta, first ? 1 : 0, st));
  if (first) GN_TRY_CUDA(cudaMemsetAsync(v_prev, 0, Pp * sizeof(double), st));
  GN_TRY_CUDA(cudaMemcpyAsync(h->hpin + 16, h->red + 256, sizeof(double), cudaMemcpyDeviceToHost, st));
  tm.mark(2);
  // 3. Delta = -(G_ema + gamma I)^{-1} g  (h->delta holds -Delta)
  int retries = 0;
  rc = damped_solve(h, G_ema, h->g, &gamma, h->delta, &retries, true);
  tm.mark(3);
  inf.chol_retries = retries;
  inf.gamma_used = gamma;
  const double h0 = 0.5 * h->hpin[16];
  inf.loss_before = inf.loss_after = h0;
  if (rc) {
    inf.status = rc;
    if (info) *info = inf;
    return rc;
  }
  if (!std::isfinite(h0)) {
    inf.status = GN_ERR_NONFINITE;
    if (info) *info = inf;
    return GN_ERR_NONFINITE;
  }
  // 4. exact curvature through J~ products, and the scalars of the 2 x 2 model
  GN_TRY_CUDA(dgemv_n(h->J, h->ldJ, R, Pp, h->delta, JD, 0.0, st));
  GN_TRY_CUDA(dgemv_n(h->J, h->ldJ, R, Pp, v_prev, Jv, 0.0, st));
  const double* xs[8] = {JD, JD, Jv, h->delta, h->delta, v_prev, h->g, h->g};
  const double* ys[8] = {JD, Jv, Jv, h->delta, v_prev, v_prev, h->delta, v_prev};
  const int64_t ns[8] = {R, R, R, Pp, Pp, Pp, Pp, Pp};
  for (int k = 0; k < 8; k++) {
    GN_TRY_CUDA(dot_partial(xs[k], ys[k], ns[k], h->red, st));
    GN_TRY_CUDA(finish_sum(h->red, h->red + 260 + k, st));
  }
  GN_TRY_CUDA(cudaMemcpyAsync(h->red + 268, h->delta + P, sizeof(double), cudaMemcpyDeviceToDevice, st));
  GN_TRY_CUDA(cudaMemcpyAsync(h->red + 269, v_prev + P, sizeof(double), cudaMemcpyDeviceToDevice, st));
  GN_TRY_CUDA(cudaMemcpyAsync(h->hpin + 20, h->red + 260, 10 * sizeof(double), cudaMemcpyDeviceToHost, st));
  GN_TRY_CUDA(cudaStreamSynchronize(st));
  const double* s = h->hpin + 20;   // with Delta = -delta:
  const double C_dd = s[0] + gamma * s[3];
  const double C_dv = -(s[1] + gamma * s[4]);
  const double C_vv = s[2] + gamma * s[5];
  const double g_d = -s[6], g_v = s[7];
  double alpha = -g_d / C_dd, mu = 0.0;
  if (!first && s[5] > 0.0) {
    const double det = C_dd * C_vv - C_dv * C_dv;
    if (det > 0.0 && std::isfinite(det)) {
      alpha = (-g_d * C_vv + g_v * C_dv) / det;
      mu = (-g_v * C_dd + g_d * C_dv) / det;
    }
  }
  const double lam_t = lam - alpha * s[8] + mu * s[9];
  // 5. the update d = alpha Delta + mu v_prev (v_prev <- d), and the loss at the new point
  GN_TRY_CUDA(ema_update(theta, h->delta, v_prev, alpha, mu, P, Pp, h->theta_t, st));
  double ht = 0.0;
  rc = residual_loss(h, h->theta_t, lam_t, h->r, &ht);
  if (rc) return rc;
  tm.mark(4);
  const double Jd2 = alpha * alpha * s[0] - 2.0 * alpha * mu * s[1] + mu * mu * s[2];
  const double model = alpha * g_d + mu * g_v + 0.5 * Jd2;   // undamped model change
  inf.alpha = alpha;
  inf.momentum = mu;
  if (!std::isfinite(ht)) {
    gamma *= 10.0;
    GN_TRY_CUDA(cudaMemsetAsync(v_prev, 0, Pp * sizeof(double), st));
    inf.status = GN_WARN_NO_DECREASE;
  } else {
    const double rho = model != 0.0 ? (ht - h0) / model : 1.0;
    if (rho < 0.25) gamma *= 1.5;
    else if (rho > 0.75) gamma *= 2.0 / 3.0;
    GN_TRY_CUDA(cudaMemcpyAsync(theta, h->theta_t, P * sizeof(double), cudaMemcpyDeviceToDevice, st));
    *lambda = lam_t;
    inf.rho = rho;
    inf.loss_after = ht;
    inf.status = GN_OK;
  }
  inf.n_trials = 1;
  *damping = gamma;
  tm.mark(5);
  GN_TRY_CUDA(cudaEventSynchronize(tm.ev[5]));
  inf.ms_phase[0] = tm.ms(0, 1);
  inf.ms_phase[1] = tm.ms(1, 2);
  inf.ms_phase[3] = tm.ms(2, 3);
  inf.ms_phase[5] = tm.ms(3, 4);
  inf.ms_phase[6] = tm.ms(0, 5);
  if (info) *info = inf;
  return inf.status;
}

}  // extern "C"
