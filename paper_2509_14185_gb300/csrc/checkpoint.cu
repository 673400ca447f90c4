// Checkpoint and resume of a fit: theta (device), lambda and the damping, with
// the equation and the architecture they belong to.  Host I/O only; the file
// layout is documented with gn_save / gn_load in include/gn.h.
#include <cstdio>
#include <cstring>
#include <vector>

#include "gn_internal.cuh"

namespace {

constexpr char kMagic[4] = {'G', 'N', 'C', 'K'};
constexpr uint32_t kVersion = 1;

#pragma pack(push, 1)   // the documented layout has no padding
struct Header {
  char magic[4];
  uint32_t version;
  int32_t equation;
  int32_t n_layers;
  int32_t widths[GN_MAX_LAYERS + 1];
  int64_t P;
  double lambda;
  double damping;
};
#pragma pack(pop)

void fill(const gn_handle* h, Header* hd) {
  memset(hd, 0, sizeof(*hd));
  memcpy(hd->magic, kMagic, 4);
  hd->version = kVersion;
  hd->equation = h->p.equation;
  hd->n_layers = h->p.n_layers;
  for (int i = 0; i <= h->p.n_layers && i <= GN_MAX_LAYERS; i++) hd->widths[i] = h->p.widths[i];
  hd->P = h->P;
}

}  // namespace

extern "C" {

int gn_save(gn_handle* h, const char* path, const double* theta, double lambda, double damping) {
  if (!h || !path || !theta) return GN_ERR_INVALID;
  Header hd;
  fill(h, &hd);
  hd.lambda = lambda;
  hd.damping = damping;
  std::vector<double> host((size_t)h->P);
  if (gn::note_cuda(cudaMemcpyAsync(host.data(), theta, (size_t)h->P * sizeof(double), cudaMemcpyDeviceToHost, h->st),
                    __FILE__, __LINE__) != cudaSuccess ||
      gn::note_cuda(cudaStreamSynchronize(h->st), __FILE__, __LINE__) != cudaSuccess)
    return GN_ERR_CUDA;
  FILE* f = fopen(path, "wb");
  if (!f) return GN_ERR_IO;
  bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 && fwrite(host.data(), sizeof(double), host.size(), f) == host.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? GN_OK : GN_ERR_IO;
}

int gn_load(gn_handle* h, const char* path, double* theta, double* lambda, double* damping) {
  if (!h || !path || !theta || !lambda || !damping) return GN_ERR_INVALID;
  FILE* f = fopen(path, "rb");
  if (!f) return GN_ERR_IO;
  Header hd, want;
  bool ok = fread(&hd, sizeof(hd), 1, f) == 1 && memcmp(hd.magic, kMagic, 4) == 0 && hd.version == kVersion;
  if (!ok) {
    fclose(f);
    return GN_ERR_IO;
  }
  fill(h, &want);
  if (hd.equation != want.equation || hd.n_layers != want.n_layers || hd.P != want.P ||
      memcmp(hd.widths, want.widths, sizeof(hd.widths)) != 0) {
    fclose(f);
    return GN_ERR_MISMATCH;
  }
  std::vector<double> host((size_t)h->P);
  ok = fread(host.data(), sizeof(double), host.size(), f) == host.size();
  fclose(f);
  if (!ok) return GN_ERR_IO;
  if (gn::note_cuda(cudaMemcpyAsync(theta, host.data(), (size_t)h->P * sizeof(double), cudaMemcpyHostToDevice, h->st),
                    __FILE__, __LINE__) != cudaSuccess ||
      gn::note_cuda(cudaStreamSynchronize(h->st), __FILE__, __LINE__) != cudaSuccess)
    return GN_ERR_CUDA;
  *lambda = hd.lambda;
  *damping = hd.damping;
  return GN_OK;
}

}  // extern "C"
