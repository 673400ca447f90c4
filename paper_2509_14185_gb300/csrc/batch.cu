// Batched profile fits (many independent GN fits of uneven size stepped
// together).  The paper sweeps lambda seeds and architectures (Methods,
// "Identifying Admissible lambda Values", funnel inference and its validation
// over seeds); each fit is an independent problem, so a batch shards with no
// exchange at all.
//
// Runtime: fits are dealt round-robin onto n_streams CUDA streams; one host
// worker thread per stream drives the damped GN steps of its fits in order
// (each step synchronises only its own stream), so the kernels of different
// fits overlap on the GPU.  Each fit keeps its own handle and workspace.
//
// Graph mode (gn_batch_capture_graph / gn_batch_graph_step): every fit's whole
// device-resident step (graph.cu) is captured as an independent branch of one
// CUDA graph, each fit on a capture stream of its own, so a batched step is one
// cudaGraphLaunch and the fits' kernel chains run concurrently with no host
// thread involved; lambda and the damping of all fits travel in one state
// array (one copy in, one copy out per step).
#include <new>
#include <thread>
#include <vector>

#include "gn_internal.cuh"

namespace gn {
int graph_prepare_fit(gn_handle* h, void* ds_slot, double* theta);
int graph_capture_fit_step(gn_handle* h, double* theta);
size_t graph_state_bytes();
void graph_host_state(gn_handle* h, double lam, double gamma, void* slot);
int graph_finish_fit(gn_handle* h, const void* slot, double* lambda, double* damping, gn_step_info* info);
}  // namespace gn

struct gn_batch {
  int n_fits;
  int n_streams;
  std::vector<cudaStream_t> streams;
  std::vector<gn_handle*> handles;
  // graph mode
  cudaStream_t origin = nullptr;          // stream the batched graph is captured on and launched into
  std::vector<cudaStream_t> cap;          // one capture stream per fit
  std::vector<cudaEvent_t> ev;            // fork (0) and one join event per fit
  unsigned char* ds = nullptr;            // device step states [n_fits]
  unsigned char* hs = nullptr;            // pinned host mirror
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {
void release_graph(gn_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}
}  // namespace

extern "C" {

int gn_batch_init(const gn_problem* problems, int n_fits, int n_streams, gn_batch** out) {
  if (!problems || !out || n_fits < 1 || n_streams < 1) return GN_ERR_INVALID;
  *out = nullptr;
  gn_batch* b = new (std::nothrow) gn_batch;
  if (!b) return GN_ERR_OOM;
  b->n_fits = n_fits;
  b->n_streams = n_streams < n_fits ? n_streams : n_fits;
  b->streams.assign(b->n_streams, nullptr);
  b->handles.assign(n_fits, nullptr);
  int rc = GN_OK;
  for (int s = 0; s < b->n_streams && rc == GN_OK; s++)
    if (cudaStreamCreateWithFlags(&b->streams[s], cudaStreamNonBlocking) != cudaSuccess) rc = GN_ERR_CUDA;
  for (int f = 0; f < n_fits && rc == GN_OK; f++)
    rc = gn_init(&problems[f], b->streams[f % b->n_streams], &b->handles[f]);
  if (rc != GN_OK) {
    gn_batch_destroy(b);
    return rc;
  }
  *out = b;
  return GN_OK;
}

int gn_batch_handle(gn_batch* b, int fit, gn_handle** out) {
  if (!b || !out || fit < 0 || fit >= b->n_fits) return GN_ERR_INVALID;
  *out = b->handles[fit];
  return GN_OK;
}

int gn_batch_step(gn_batch* b, double* const* thetas, double* lambdas, double* dampings, gn_step_info* infos,
                  int* status) {
  if (!b || !thetas || !lambdas || !dampings) return GN_ERR_INVALID;
  std::vector<int> rcs(b->n_fits, GN_OK);
  int dev = 0;
  cudaGetDevice(&dev);
  auto worker = [&](int s) {
    cudaSetDevice(dev);
    for (int f = s; f < b->n_fits; f += b->n_streams)
      rcs[f] = gn_step(b->handles[f], thetas[f], &lambdas[f], &dampings[f], infos ? &infos[f] : nullptr);
  };
  std::vector<std::thread> pool;
  for (int s = 1; s < b->n_streams; s++) pool.emplace_back(worker, s);
  worker(0);
  for (auto& t : pool) t.join();
  int worst = GN_OK;
  for (int f = 0; f < b->n_fits; f++) {
    if (status) status[f] = rcs[f];
    if (rcs[f] < worst) worst = rcs[f];
  }
  return worst;   // GN_OK, or the most negative error of any fit (warnings are per fit)
}

int gn_batch_capture_graph(gn_batch* b, double* const* thetas) {
  if (!b || !thetas) return GN_ERR_INVALID;
  for (int f = 0; f < b->n_fits; f++)
    if (!thetas[f]) return GN_ERR_INVALID;
  release_graph(b);
  const size_t sb = gn::graph_state_bytes();
  if (!b->ds) {
    if (GN_NOTE(cudaMalloc((void**)&b->ds, sb * b->n_fits)) != cudaSuccess) return GN_ERR_OOM;
    if (GN_NOTE(cudaMallocHost((void**)&b->hs, sb * b->n_fits)) != cudaSuccess) return GN_ERR_OOM;
    if (GN_NOTE(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking)) != cudaSuccess) return GN_ERR_CUDA;
    b->cap.assign(b->n_fits, nullptr);
    b->ev.assign(b->n_fits + 1, nullptr);
    for (int f = 0; f < b->n_fits; f++)
      if (GN_NOTE(cudaStreamCreateWithFlags(&b->cap[f], cudaStreamNonBlocking)) != cudaSuccess) return GN_ERR_CUDA;
    for (auto& e : b->ev)
      if (GN_NOTE(cudaEventCreateWithFlags(&e, cudaEventDisableTiming)) != cudaSuccess) return GN_ERR_CUDA;
  }
  // per fit: state slot, workspace sized for capture, the retry ("solve") graph
  for (int f = 0; f < b->n_fits; f++) {
    const int rc = gn::graph_prepare_fit(b->handles[f], b->ds + sb * f, thetas[f]);
    if (rc) return rc;
  }
  if (GN_NOTE(cudaDeviceSynchronize()) != cudaSuccess) return GN_ERR_CUDA;
  if (GN_NOTE(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return GN_ERR_CUDA;
  int rc = GN_OK;
  if (GN_NOTE(cudaEventRecord(b->ev[0], b->origin)) != cudaSuccess) rc = GN_ERR_CUDA;
  for (int f = 0; f < b->n_fits && rc == GN_OK; f++) {
    gn_handle* h = b->handles[f];
    cudaStream_t saved = h->st;
    h->st = b->cap[f];
    if (GN_NOTE(cudaStreamWaitEvent(h->st, b->ev[0], 0)) != cudaSuccess) rc = GN_ERR_CUDA;
    if (rc == GN_OK) rc = gn::graph_capture_fit_step(h, thetas[f]);
    if (rc == GN_OK && GN_NOTE(cudaEventRecord(b->ev[f + 1], h->st)) != cudaSuccess) rc = GN_ERR_CUDA;
    if (rc == GN_OK && GN_NOTE(cudaStreamWaitEvent(b->origin, b->ev[f + 1], 0)) != cudaSuccess) rc = GN_ERR_CUDA;
    h->st = saved;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = GN_NOTE(cudaStreamEndCapture(b->origin, &g));
  if (rc != GN_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != GN_OK ? rc : GN_ERR_CUDA;
  }
  b->graph = g;
  if (GN_NOTE(cudaGraphInstantiate(&b->exec, g, cudaGraphInstantiateFlagUseNodePriority)) != cudaSuccess) {
    release_graph(b);
    return GN_ERR_CUDA;
  }
  return GN_OK;
}

int gn_batch_graph_step(gn_batch* b, double* lambdas, double* dampings, gn_step_info* infos, int* status) {
  if (!b || !lambdas || !dampings) return GN_ERR_INVALID;
  if (!b->exec) return GN_ERR_INVALID;   // gn_batch_capture_graph first
  const size_t sb = gn::graph_state_bytes();
  for (int f = 0; f < b->n_fits; f++) gn::graph_host_state(b->handles[f], lambdas[f], dampings[f], b->hs + sb * f);
  if (GN_NOTE(cudaMemcpyAsync(b->ds, b->hs, sb * b->n_fits, cudaMemcpyHostToDevice, b->origin)) != cudaSuccess ||
      GN_NOTE(cudaGraphLaunch(b->exec, b->origin)) != cudaSuccess ||
      GN_NOTE(cudaMemcpyAsync(b->hs, b->ds, sb * b->n_fits, cudaMemcpyDeviceToHost, b->origin)) != cudaSuccess ||
      GN_NOTE(cudaStreamSynchronize(b->origin)) != cudaSuccess)
    return GN_ERR_CUDA;
  int worst = GN_OK;
  for (int f = 0; f < b->n_fits; f++) {
    const int rc = gn::graph_finish_fit(b->handles[f], b->hs + sb * f, &lambdas[f], &dampings[f],
                                        infos ? &infos[f] : nullptr);
    if (status) status[f] = rc;
    if (rc < worst) worst = rc;
  }
  return worst;
}

int gn_batch_destroy(gn_batch* b) {
  if (!b) return GN_OK;
  release_graph(b);
  for (auto* h : b->handles)
    if (h) gn_destroy(h);
  for (auto s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (auto s : b->cap)
    if (s) cudaStreamDestroy(s);
  for (auto e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->ds) cudaFree(b->ds);
  if (b->hs) cudaFreeHost(b->hs);
  delete b;
  return GN_OK;
}

}  // extern "C"
