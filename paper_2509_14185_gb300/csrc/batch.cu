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
#include <new>
#include <thread>
#include <vector>

#include "gn_internal.cuh"

struct gn_batch {
  int n_fits;
  int n_streams;
  std::vector<cudaStream_t> streams;
  std::vector<gn_handle*> handles;
};

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

int gn_batch_destroy(gn_batch* b) {
  if (!b) return GN_OK;
  for (auto* h : b->handles)
    if (h) gn_destroy(h);
  for (auto s : b->streams)
    if (s) cudaStreamDestroy(s);
  delete b;
  return GN_OK;
}

}  // extern "C"
