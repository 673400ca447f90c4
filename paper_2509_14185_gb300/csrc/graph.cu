// Device-resident damped Gauss-Newton step, captured once as a CUDA graph and
// replayed (Methods, "Second-order Optimizer": the same step as gn_step).
//
// gn_step decides three things on the host between launches: whether the
// factorisation of G + gamma I succeeded, which line-search trial is accepted,
// and the new damping.  Here those decisions run in one-thread kernels on a
// device-resident state (StepState), so one step is a fixed launch sequence:
//
//   graph "step"  = rows + Jacobian + Gram + g + loss, then the "solve" part;
//                   under SPLIT_ALL (one row block) the Gram runs as column-major
//                   chunks on a low-priority stream and the factorisation starts
//                   each 256-column strip as soon as its columns are in A
//                   (the pipelined step: same arithmetic, overlapped schedule)
//   graph "solve" = G + gamma I, factorisation, triangular solves, the model
//                   scalars, eight conditional IF nodes in sequence whose
//                   bodies are the Armijo trials (theta_t = theta - alpha delta,
//                   residual-only pass, loss, acceptance test, which enables the
//                   next trial only after a rejection), and the commit (theta,
//                   lambda, LM damping update).  The trial count is bounded by
//                   the graph's structure, not by a loop condition.
//
// lambda and gamma live in the state, read by the kernels through pointers, so
// a graph is independent of their values; theta is fixed per graph (its device
// address is a kernel parameter).  A failed factorisation ends the graph with
// status kNeedRetry; the host then raises gamma x10 and replays only the
// "solve" graph (at most 5 times), which is gn_step's escalation rule.
//
// Batches: every fit's "step" part is captured into one graph as an
// independent branch (its own capture stream), so one cudaGraphLaunch runs a
// whole batched step; fits that need a retry replay their own "solve" graph.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "gn_internal.cuh"

namespace gn {

struct StepState {
  double lam, gamma;        // in: current lambda and damping; out: updated
  double lam_t, alpha;      // current trial
  double h0, gd, dGd, dlam; // loss and model scalars of the step
  double ht, rho;           // accepted trial loss, LM ratio
  double gamma_used;        // damping of the factorisation the step used
  double max_res;           // max |R_k| over the interior points at the step's starting point
  int n_trials, accepted, status, pad;
};

constexpr int kNeedRetry = 100;   // internal: the factorisation failed, raise gamma and solve again
constexpr int kMaxTrials = 8;     // Armijo trials (gn_step's limit)

struct GraphState {
  StepState* ds = nullptr;        // device state (owned unless it lives in a batch array)
  bool ds_owned = false;
  StepState* hs = nullptr;        // pinned host mirror
  const double* theta = nullptr;  // parameters the graphs were captured for
  cudaGraph_t g_step = nullptr, g_solve = nullptr;
  cudaGraphExec_t x_step = nullptr, x_solve = nullptr;
  cudaStream_t body = nullptr;    // capture stream of the line-search bodies
  cudaStream_t body_aux = nullptr;   // the bodies' side stream (the handle's own st_aux has
                                     // joined the step's capture, a sequence of its own)
  cudaStream_t gst = nullptr;     // stream the graphs are captured on and launched into (the
                                  // handle's own stream may be the legacy default stream,
                                  // which cannot be captured)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_in = nullptr;
  // phase marks recorded inside the handle's own graphs (external event nodes): 0 start,
  // 1 Jacobian done, 2 Gram and gradient done, 4 factorisation start, 5 solves done,
  // 6 model scalars done, 7 commit done; 3 is unused
  cudaEvent_t evp[8] = {};
  bool marks = false;   // the graphs carry the marks (one row block; not a batch branch)
  int precision = -1, n_slices = -1, lam_frozen = -1, staged = -1, pipe = -2;   // of the handle when captured
  double stage_eps = 0.0;
  // kernels per replay, for gn_kernel_launches: outside the trial bodies (step graph, solve
  // graph, a batch's step branch) and per line-search trial that runs
  long long k_step = 0, k_solve = 0, k_branch = 0, k_trial = 0;
};

namespace {

#define GN_G_TRY(x)                                         \
  do {                                                      \
    cudaError_t e_ = GN_NOTE(x);                            \
    if (e_ != cudaSuccess) return GN_ERR_CUDA;              \
  } while (0)

// Model scalars after the solve (red[256] = |r~|^2, red[257] = g.delta, red[258] =
// delta.G.delta, delta[P] = the lambda component); decides whether the line search runs.
__global__ void model_kernel(const double* __restrict__ red, const double* __restrict__ delta, int64_t P,
                             const int* __restrict__ flag, StepState* s, cudaGraphConditionalHandle first) {
  s->n_trials = 0;
  s->accepted = 0;
  s->alpha = 1.0;
  s->rho = 0.0;
  s->gamma_used = s->gamma;
  s->h0 = 0.5 * red[256];
  s->ht = s->h0;
  s->gd = red[257];
  s->dGd = red[258];
  s->dlam = delta[P];
  s->max_res = red[kMaxResSlot];
  int status = GN_OK;
  if (flag[2] & 2) status = GN_ERR_TIMEOUT;          // a bounded tensor-core wait gave up
  else if (!isfinite(s->h0)) status = GN_ERR_NONFINITE;   // before the pivots: no retries on NaN rows
  else if (flag[1]) status = kNeedRetry;             // a pivot was not positive
  s->status = status;
  cudaGraphSetConditional(first, status == GN_OK ? 1u : 0u);   // run the first trial?
}

// theta_t = theta - alpha delta, lambda_t = lambda - alpha delta_P (alpha a power of two,
// so both products are exact and the result is that of gn_step's trial).
__global__ void trial_kernel(const double* __restrict__ theta, const double* __restrict__ delta, int64_t P,
                             double* theta_t, StepState* s) {
  const double alpha = s->alpha;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
    theta_t[i] = theta[i] - alpha * delta[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) s->lam_t = s->lam - alpha * s->dlam;
}

// Armijo test of the trial just evaluated (c1 = 1e-4, alpha halved after a rejection);
// `next` is the condition of the following trial's IF node (none after the last trial).
__global__ void armijo_kernel(const double* __restrict__ red, StepState* s, cudaGraphConditionalHandle next,
                              int has_next) {
  const double ht = 0.5 * red[256];
  const double alpha = s->alpha;
  s->n_trials = s->n_trials + 1;
  s->ht = ht;
  const bool ok = isfinite(ht) && ht <= s->h0 - 1e-4 * alpha * s->gd;
  if (ok) s->accepted = 1;
  else s->alpha = 0.5 * alpha;
  if (has_next) cudaGraphSetConditional(next, ok ? 0u : 1u);
}

// Accepted: theta = theta_t (all threads), lambda and the LM damping update (one thread).
// Rejected: damping x10.  The status stays as the model kernel left it otherwise.
__global__ void commit_kernel(double* theta, const double* __restrict__ theta_t, int64_t P, StepState* s) {
  if (s->status != GN_OK) return;
  const bool acc = s->accepted != 0;
  if (acc)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
      theta[i] = theta_t[i];
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  if (acc) {
    const double a = s->alpha;
    const double pred = a * s->gd - 0.5 * a * a * s->dGd;
    const double rho = pred != 0.0 ? (s->h0 - s->ht) / pred : 1.0;
    double gamma = s->gamma;
    if (rho < 0.25) gamma *= 1.5;
    else if (rho > 0.75) gamma *= 2.0 / 3.0;
    s->gamma = gamma;
    s->rho = rho;
    s->lam = s->lam_t;
  } else {
    s->gamma *= 10.0;
    s->status = GN_WARN_NO_DECREASE;
  }
}

unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 2048) b = 2048;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// Rows, Jacobian (row blocks), Gram and gradient, loss: the first half of gn_step.
// An external event node marking a phase boundary (only in graphs that carry the marks).
int mark(gn_handle* h, bool on, int k) {
  if (on) GN_G_TRY(cudaEventRecordWithFlags(h->gs->evp[k], h->st, cudaEventRecordExternal));
  return GN_OK;
}

int capture_rows_gram(gn_handle* h, const double* theta, bool marks) {
  GraphState* gs = h->gs;
  cudaStream_t st = h->st;
  GN_G_TRY(cudaMemsetAsync(h->flag + 2, 0, sizeof(int), st));
  const int64_t nblk = (h->n_rows + h->jrows - 1) / h->jrows;
  marks = marks && nblk == 1;
  int rc = mark(h, marks, 0);
  for (int64_t b = 0; b < nblk && !rc; b++) {
    const int64_t lo = b * h->jrows;
    const int64_t hi = (lo + h->jrows < h->n_rows) ? lo + h->jrows : h->n_rows;
    Pass ps = {MODE_JACOBIAN, h->r, h->J, h->ldJ, lo, hi, nullptr, &gs->ds->lam};
    rc = run_pass(h, theta, 0.0, ps, nullptr);
    if (!rc) rc = mark(h, marks, 1);
    if (!rc) rc = gram_into(h, h->J, h->ldJ, hi - lo, h->r + lo, h->G, h->g, h->precision, b > 0);
    if (!rc) rc = mark(h, marks, 2);
  }
  if (rc) return rc;
  rc = loss_of(h, h->r, 0);
  return rc ? rc : max_res_of(h, h->r);
}

// The second half: damped factorisation and solve, model scalars, IF(trial) x 8, commit.
// gate (pipelined step): A's strips are copied by the Gram's stream, which signals each strip
// through its gate event and the whole Gram (with G's mirror) through join.
int capture_solve(gn_handle* h, double* theta, bool marks, const cudaEvent_t* gate = nullptr,
                  cudaEvent_t join = nullptr) {
  GraphState* gs = h->gs;
  cudaStream_t st = h->st;
  const int64_t Pp = h->Pp, P = h->P;
  StepState* ds = gs->ds;
  // the line search: kMaxTrials IF nodes in sequence, trial t runs when the previous kernel
  // (the model kernel for t = 0, trial t - 1's Armijo kernel otherwise) set its condition;
  // the conditions default to 0 at every launch, so the graph can never run more trials
  cudaStreamCaptureStatus cs;
  cudaGraph_t cg = nullptr;
  GN_G_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive) return GN_ERR_CUDA;
  cudaGraphConditionalHandle cond[kMaxTrials];
  for (int t = 0; t < kMaxTrials; t++)
    GN_G_TRY(cudaGraphConditionalHandleCreate(&cond[t], cg, 0, cudaGraphCondAssignDefault));

  if (mark(h, marks, 4)) return GN_ERR_CUDA;
  if (!gate) {
    GN_G_TRY(copy_add_diag(h->G, h->A, Pp, Pp, 0.0, &ds->gamma, st));   // gamma from the step state
  }
  GN_G_TRY(cudaMemsetAsync(h->flag + 1, 0, sizeof(int), st));
  if (h->precision == GN_PREC_SPLIT_ALL) {
    int rc = GN_OK;
    cudaError_t e = cholesky_factor_split(h, h->A, Pp, Pp, h->Linv, h->flag + 1, h->n_slices, h->g, h->vtmp + Pp,
                                          h->vtmp, &rc, gate);
    if (rc) return rc;
    GN_G_TRY(e);
    GN_G_TRY(cholesky_solve_backward(h->A, Pp, Pp, h->Linv, h->vtmp + Pp, h->delta, h->vtmp, st));
  } else {
    GN_G_TRY(cholesky_factor(h->A, Pp, Pp, h->Linv, h->flag + 1, st));
    GN_G_TRY(cholesky_solve(h->A, Pp, Pp, h->Linv, h->g, h->delta, h->vtmp, st));
  }
  if (mark(h, marks, 5)) return GN_ERR_CUDA;
  if (join) GN_G_TRY(cudaStreamWaitEvent(st, join, 0));   // the model reads all of G
  GN_G_TRY(dot_partial(h->g, h->delta, Pp, h->red, st));
  GN_G_TRY(finish_sum(h->red, h->red + 257, st));
  GN_G_TRY(quad_lower(h->G, Pp, Pp, h->delta, h->vtmp, st));   // delta.G.delta from the lower triangle
  GN_G_TRY(dot_partial(h->delta, h->vtmp, Pp, h->red, st));
  GN_G_TRY(finish_sum(h->red, h->red + 258, st));
  model_kernel<<<1, 1, 0, st>>>(h->red, h->delta, P, h->flag, ds, cond[0]);
  count_launch();
  GN_G_TRY(cudaGetLastError());
  if (mark(h, marks, 6)) return GN_ERR_CUDA;

  for (int t = 0; t < kMaxTrials; t++) {
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    GN_G_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, nullptr, &ndeps));
    // (the parameter struct has no usable default constructor: zeroed raw storage instead)
    alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
    memset(npbuf, 0, sizeof(npbuf));
    cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(npbuf);
    np->type = cudaGraphNodeTypeConditional;
    np->conditional.handle = cond[t];
    np->conditional.type = cudaGraphCondTypeIf;
    np->conditional.size = 1;
    cudaGraphNode_t inode;
    GN_G_TRY(cudaGraphAddNode(&inode, cg, deps, nullptr, ndeps, np));
    cudaGraph_t body = np->conditional.phGraph_out[0];
    GN_G_TRY(cudaStreamUpdateCaptureDependencies(st, &inode, nullptr, 1, cudaStreamSetCaptureDependencies));
    // the body: one trial, captured on the body stream
    GN_G_TRY(cudaStreamBeginCaptureToGraph(gs->body, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const long long k0 = g_launches.load();
    h->st = gs->body;
    cudaStream_t aux_saved = h->st_aux;
    if (h->st_aux) h->st_aux = gs->body_aux;   // a side stream that no other capture holds
    trial_kernel<<<grid_for(P), 256, 0, gs->body>>>(theta, h->delta, P, h->theta_t, ds);
    count_launch();
    int rc = GN_NOTE(cudaGetLastError()) == cudaSuccess ? GN_OK : GN_ERR_CUDA;
    if (!rc) {
      Pass ps = {MODE_RESIDUAL, h->r, nullptr, 0, 0, 0, nullptr, &ds->lam_t};
      rc = run_pass(h, h->theta_t, 0.0, ps, nullptr);
    }
    if (!rc) rc = loss_of(h, h->r, 0);
    if (!rc) {
      const bool has_next = t + 1 < kMaxTrials;
      armijo_kernel<<<1, 1, 0, gs->body>>>(h->red, ds, has_next ? cond[t + 1] : cond[t], has_next ? 1 : 0);
      count_launch();
      if (GN_NOTE(cudaGetLastError()) != cudaSuccess) rc = GN_ERR_CUDA;
    }
    h->st = st;
    h->st_aux = aux_saved;
    gs->k_trial = g_launches.load() - k0;
    cudaGraph_t out = nullptr;
    const cudaError_t ee = GN_NOTE(cudaStreamEndCapture(gs->body, &out));
    if (rc) return rc;
    if (ee != cudaSuccess) return GN_ERR_CUDA;
  }
  commit_kernel<<<grid_for(P), 256, 0, st>>>(theta, h->theta_t, P, ds);
  count_launch();
  GN_G_TRY(cudaGetLastError());
  return mark(h, marks, 7);
}

// The pipelined step (one row block, SPLIT_ALL): rows and Jacobian; then the Gram as column
// chunks on the lowest-priority stream, which copies each finished 256-column strip into
// A = G + gamma I and signals it; the factorisation starts each strip at its signal.  The
// gradient and the loss run on the capture stream beside the first chunks.
int capture_pipelined(gn_handle* h, double* theta, bool marks, int64_t chunk) {
  GraphState* gs = h->gs;
  cudaStream_t st = h->st;
  GN_G_TRY(cudaMemsetAsync(h->flag + 2, 0, sizeof(int), st));
  int rc = mark(h, marks, 0);
  Pass ps = {MODE_JACOBIAN, h->r, h->J, h->ldJ, 0, h->n_rows, nullptr, &gs->ds->lam};
  if (!rc) rc = run_pass(h, theta, 0.0, ps, nullptr);
  if (!rc) rc = mark(h, marks, 1);
  if (rc) return rc;
  GN_G_TRY(ensure_chol_streams(h));
  std::vector<cudaEvent_t> events, gate;
  struct Guard {   // captured dependencies are edges of the graph: the events can go afterwards
    std::vector<cudaEvent_t>& v;
    ~Guard() {
      for (auto e : v)
        if (e) cudaEventDestroy(e);
    }
  } guard{events};
  cudaStream_t sg = h->st_g;
  rc = split_gram_pipelined(h, h->J, h->ldJ, h->n_rows, h->G, h->A, &gs->ds->gamma, chunk, st, sg, events, gate);
  if (rc) return rc;
  if (marks) GN_G_TRY(cudaEventRecordWithFlags(gs->evp[2], sg, cudaEventRecordExternal));
  cudaEvent_t join = nullptr;
  GN_G_TRY(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
  events.push_back(join);
  GN_G_TRY(cudaEventRecord(join, sg));
  GN_G_TRY(dgemv_t_scratch(h->J, h->ldJ, h->n_rows, h->Pp, h->r, h->g, 0.0, h->vtmp, st));
  rc = loss_of(h, h->r, 0);
  if (!rc) rc = max_res_of(h, h->r);
  if (rc) return rc;
  return capture_solve(h, theta, marks, gate.data(), join);
}

// Capture one graph on h->st: the whole step (with_rows) or the solve part only.
int capture(gn_handle* h, double* theta, bool with_rows, cudaGraph_t* out) {
  *out = nullptr;
  const int64_t chunk = with_rows ? pipeline_chunk_tiles(h) : 0;   // (queries the device: before capture)
  GN_G_TRY(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
  h->capturing = 1;
  const long long k0 = g_launches.load();
  const bool marks = h->gs->marks;
  int rc = GN_OK;
  if (chunk > 0) {
    rc = capture_pipelined(h, theta, marks, chunk);
  } else {
    rc = with_rows ? capture_rows_gram(h, theta, marks) : GN_OK;
    if (!rc) rc = capture_solve(h, theta, marks);
  }
  // capture counted each launch once; replays add what actually runs
  const long long k = g_launches.load() - k0;
  g_launches.fetch_sub(k);
  (with_rows ? h->gs->k_step : h->gs->k_solve) = k - kMaxTrials * h->gs->k_trial;
  h->capturing = 0;
  cudaGraph_t g = nullptr;
  const cudaError_t e = GN_NOTE(cudaStreamEndCapture(h->st, &g));
  if (rc || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc ? rc : GN_ERR_CUDA;
  }
  *out = g;
  return GN_OK;
}

void destroy_graphs(GraphState* gs) {
  if (gs->x_step) cudaGraphExecDestroy(gs->x_step);
  if (gs->x_solve) cudaGraphExecDestroy(gs->x_solve);
  if (gs->g_step) cudaGraphDestroy(gs->g_step);
  if (gs->g_solve) cudaGraphDestroy(gs->g_solve);
  gs->x_step = gs->x_solve = nullptr;
  gs->g_step = gs->g_solve = nullptr;
  gs->theta = nullptr;
}

// Per-handle graph state (device state, pinned mirror, streams, timing events).
int ensure_state(gn_handle* h, StepState* external_ds) {
  if (!h->gs) {
    GraphState* gs = new (std::nothrow) GraphState;
    if (!gs) return GN_ERR_OOM;
    h->gs = gs;
    if (GN_NOTE(cudaMallocHost((void**)&gs->hs, sizeof(StepState))) != cudaSuccess) return GN_ERR_OOM;
    memset(gs->hs, 0, sizeof(StepState));
    GN_G_TRY(cudaStreamCreateWithFlags(&gs->body, cudaStreamNonBlocking));
    int least = 0, greatest = 0;
    GN_G_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    GN_G_TRY(cudaStreamCreateWithPriority(&gs->body_aux, cudaStreamNonBlocking, greatest));
    GN_G_TRY(cudaStreamCreateWithFlags(&gs->gst, cudaStreamNonBlocking));
    GN_G_TRY(cudaEventCreate(&gs->ev0));
    GN_G_TRY(cudaEventCreate(&gs->ev1));
    GN_G_TRY(cudaEventCreateWithFlags(&gs->ev_in, cudaEventDisableTiming));
    for (auto& e : gs->evp) GN_G_TRY(cudaEventCreate(&e));
  }
  GraphState* gs = h->gs;
  if (external_ds) {
    if (gs->ds != external_ds) {
      destroy_graphs(gs);
      if (gs->ds_owned) cudaFree(gs->ds);
      gs->ds = external_ds;
      gs->ds_owned = false;
    }
  } else if (!gs->ds) {
    if (GN_NOTE(cudaMalloc((void**)&gs->ds, sizeof(StepState))) != cudaSuccess) return GN_ERR_OOM;
    gs->ds_owned = true;
  }
  return GN_OK;
}

// (Re)build the graphs of a handle for parameters theta.  with_step = false builds only
// the solve graph (a batch holds the step part in its own graph).
int build_graphs(gn_handle* h, double* theta, bool with_step) {
  GraphState* gs = h->gs;
  destroy_graphs(gs);
  gs->marks = with_step;   // a batch fit's retry graph carries none
  int rc = prepare_for_capture(h);
  if (rc) return rc;
  GN_G_TRY(cudaStreamSynchronize(h->st));   // nothing of an earlier eager call may be in flight
  cudaStream_t saved = h->st;
  h->st = gs->gst;
  if (with_step) rc = capture(h, theta, true, &gs->g_step);
  if (!rc) rc = capture(h, theta, false, &gs->g_solve);
  h->st = saved;
  if (rc) return rc;
  // per-node priorities keep the factorisation's look-ahead split (critical path high)
  if (with_step) GN_G_TRY(cudaGraphInstantiate(&gs->x_step, gs->g_step, cudaGraphInstantiateFlagUseNodePriority));
  GN_G_TRY(cudaGraphInstantiate(&gs->x_solve, gs->g_solve, cudaGraphInstantiateFlagUseNodePriority));
  gs->theta = theta;
  gs->precision = h->precision;
  gs->n_slices = h->n_slices;
  gs->lam_frozen = h->lam_frozen;
  gs->staged = h->staged;
  gs->stage_eps = h->stage_eps;
  gs->pipe = h->pipe_tiles;
  return GN_OK;
}

// After the step graph ran and gs->hs holds the device state: retries of the solve graph
// (gamma x10, at most 5) and the step's results.  Synchronises.
int finish_step(gn_handle* h, double* lambda, double* damping, gn_step_info* info, int retries_done) {
  GraphState* gs = h->gs;
  StepState* s = gs->hs;
  int retries = retries_done;
  while (s->status == kNeedRetry) {
    if (retries == 5) break;
    s->gamma *= 10.0;
    retries++;
    GN_G_TRY(cudaMemcpyAsync(gs->ds, s, sizeof(StepState), cudaMemcpyHostToDevice, gs->gst));
    GN_G_TRY(cudaGraphLaunch(gs->x_solve, gs->gst));
    GN_G_TRY(cudaMemcpyAsync(s, gs->ds, sizeof(StepState), cudaMemcpyDeviceToHost, gs->gst));
    GN_G_TRY(cudaStreamSynchronize(gs->gst));
    count_launch((int)(gs->k_solve + gs->k_trial * s->n_trials));
  }
  gn_step_info inf;
  memset(&inf, 0, sizeof(inf));
  inf.chol_retries = retries;
  inf.max_abs_res = s->max_res;
  int status = s->status;
  if (status == kNeedRetry) status = GN_ERR_NOT_SPD;
  // the damping of the accepted factorisation (before the LM update), as gn_step reports it
  inf.gamma_used = s->gamma_used;
  if (status == GN_OK) {
    inf.loss_before = s->h0;
    inf.loss_after = s->ht;
    inf.alpha = s->alpha;
    inf.rho = s->rho;
    inf.n_trials = s->n_trials;
    *lambda = s->lam;
    *damping = s->gamma;
  } else if (status == GN_WARN_NO_DECREASE) {
    inf.loss_before = s->h0;
    inf.loss_after = s->h0;
    inf.n_trials = s->n_trials;
    *damping = s->gamma;
  } else if (status == GN_ERR_NONFINITE) {
    inf.loss_before = s->h0;
    inf.loss_after = s->h0;
  }
  inf.status = status;
  if (info) *info = inf;
  if (status == GN_ERR_TIMEOUT) set_detail(__FILE__, __LINE__, "a bounded wait in a tensor-core kernel timed out");
  return status;
}

}  // namespace

void graph_release(gn_handle* h) {
  GraphState* gs = h->gs;
  if (!gs) return;
  destroy_graphs(gs);
  if (gs->ds_owned && gs->ds) cudaFree(gs->ds);
  if (gs->hs) cudaFreeHost(gs->hs);
  if (gs->body) cudaStreamDestroy(gs->body);
  if (gs->body_aux) cudaStreamDestroy(gs->body_aux);
  if (gs->gst) cudaStreamDestroy(gs->gst);
  if (gs->ev_in) cudaEventDestroy(gs->ev_in);
  if (gs->ev0) cudaEventDestroy(gs->ev0);
  if (gs->ev1) cudaEventDestroy(gs->ev1);
  for (auto e : gs->evp)
    if (e) cudaEventDestroy(e);
  delete gs;
  h->gs = nullptr;
}

// Batch support (batch.cu): state slots and graphs of the fits.
int graph_prepare_fit(gn_handle* h, void* ds_slot, double* theta) {
  int rc = ensure_state(h, static_cast<StepState*>(ds_slot));
  if (rc) return rc;
  return build_graphs(h, theta, false);
}
// The step part of one fit, captured on h->st (which the batch has made part of its capture).
int graph_capture_fit_step(gn_handle* h, double* theta) {
  h->capturing = 1;
  const long long k0 = g_launches.load();
  int rc = capture_rows_gram(h, theta, false);
  if (!rc) rc = capture_solve(h, theta, false);
  const long long k = g_launches.load() - k0;
  g_launches.fetch_sub(k);
  h->gs->k_branch = k - kMaxTrials * h->gs->k_trial;
  h->capturing = 0;
  return rc;
}
size_t graph_state_bytes() { return sizeof(StepState); }
void graph_host_state(gn_handle* h, double lam, double gamma, void* slot) {
  (void)h;
  StepState s;
  memset(&s, 0, sizeof(s));
  s.lam = lam;
  s.gamma = gamma;
  memcpy(slot, &s, sizeof(s));
}
int graph_finish_fit(gn_handle* h, const void* slot, double* lambda, double* damping, gn_step_info* info) {
  memcpy(h->gs->hs, slot, sizeof(StepState));
  count_launch((int)(h->gs->k_branch + h->gs->k_trial * h->gs->hs->n_trials));
  return finish_step(h, lambda, damping, info, 0);
}

}  // namespace gn

using namespace gn;

extern "C" {

int gn_step_graph(gn_handle* h, double* theta, double* lambda, double* damping, gn_step_info* info) {
  if (!h || !theta || !lambda || !damping) return GN_ERR_INVALID;
  int rc = ensure_state(h, nullptr);
  if (rc) return rc;
  GraphState* gs = h->gs;
  if (gs->theta != theta || !gs->x_step || gs->precision != h->precision || gs->n_slices != h->n_slices ||
      gs->lam_frozen != h->lam_frozen || gs->staged != h->staged || gs->stage_eps != h->stage_eps ||
      gs->pipe != h->pipe_tiles) {
    rc = build_graphs(h, theta, true);
    if (rc) return rc;
  }
  StepState* s = gs->hs;
  memset(s, 0, sizeof(*s));
  s->lam = *lambda;
  s->gamma = *damping;
  // the graphs run on their own stream, after everything queued on the handle's stream
  GN_G_TRY(cudaEventRecord(gs->ev_in, h->st));
  GN_G_TRY(cudaStreamWaitEvent(gs->gst, gs->ev_in, 0));
  GN_G_TRY(cudaMemcpyAsync(gs->ds, s, sizeof(StepState), cudaMemcpyHostToDevice, gs->gst));
  GN_G_TRY(cudaEventRecord(gs->ev0, gs->gst));
  GN_G_TRY(cudaGraphLaunch(gs->x_step, gs->gst));
  GN_G_TRY(cudaMemcpyAsync(s, gs->ds, sizeof(StepState), cudaMemcpyDeviceToHost, gs->gst));
  GN_G_TRY(cudaStreamSynchronize(gs->gst));
  count_launch((int)(gs->k_step + gs->k_trial * s->n_trials));
  gn_step_info inf;
  const int status = finish_step(h, lambda, damping, &inf, 0);
  GN_G_TRY(cudaEventRecord(gs->ev1, gs->gst));
  GN_G_TRY(cudaEventSynchronize(gs->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, gs->ev0, gs->ev1);
  inf.ms_phase[6] = ms;
  if (gs->marks && (h->n_rows + h->jrows - 1) / h->jrows == 1) {
    auto el = [&](int a, int b) {
      float v = 0.f;
      return cudaEventElapsedTime(&v, gs->evp[a], gs->evp[b]) == cudaSuccess ? (double)v : 0.0;
    };
    inf.ms_phase[0] = el(0, 1);   // Jacobian
    inf.ms_phase[1] = el(1, 2);   // Gram and gradient
    if (inf.status != GN_ERR_NOT_SPD) {
      inf.ms_phase[3] = el(4, 5);   // damped factorisation and solves (the last replay)
      inf.ms_phase[4] = el(5, 6);   // model scalars
      inf.ms_phase[5] = el(6, 7);   // line search and commit
    }
  }
  if (info) *info = inf;
  return status;
}

}  // extern "C"
