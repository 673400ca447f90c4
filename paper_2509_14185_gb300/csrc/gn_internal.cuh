// Internal declarations of libgn: handle layout, network descriptor and the
// device launchers shared between translation units.  Nothing here is part
// of the public ABI (include/gn.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <vector>
#include <stdint.h>

#include <atomic>

#include "../../include/gn.h"

namespace gn {

constexpr int kWarp = 32;

// Kernels launched by this library in this process (diagnostic, gn_kernel_launches).
extern std::atomic<long long> g_launches;
inline void count_launch(int n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Description of the last failing CUDA call on this host thread (gn_last_error_detail).
void set_detail(const char* where, int line, const char* what);
cudaError_t note_cuda(cudaError_t e, const char* where, int line);
#define GN_NOTE(x) ::gn::note_cuda((x), __FILE__, __LINE__)

// Kinds of "points" whose rows the jet kernel produces.
enum PointKind : int {
  KIND_INTERIOR = 0,  // interior collocation point: N_E residual rows
  KIND_WALL = 1,      // wall point (2D): one row, the stream function value
  KIND_NORM = 2,      // normalisation point: one row
  KIND_NODE = 3,      // CCF Hilbert node: one row, g = Theta / y at the node
  KIND_PROBE = 4,     // field jets at a point: per field value, gradient, Hessian (2D) into r
  KIND_INF = 5,       // decay point of the data loss: one row, the value of field 0
  KIND_RELU = 6       // bound point of the data loss: one row, relu(s (Phi_A0 - b))
};

enum JetMode : int { MODE_RESIDUAL = 0, MODE_JACOBIAN = 1, MODE_GRADIENT = 2 };

// Values the probe kind writes per point: per field value, gradient and Hessian (1D: one
// zero in place of the Hessian), then for CCF the value of g = Theta / y.
inline int probe_ld(int eq, int d, int nf) { return nf * (1 + d + (d == 1 ? 1 : 3)) + (eq == GN_CCF ? 1 : 0); }

struct NetDesc {
  int L;                            // linear layers
  int w[GN_MAX_LAYERS + 1];         // widths
  int64_t offW[GN_MAX_LAYERS];      // W_l offset in theta (out x in, row-major)
  int64_t offB[GN_MAX_LAYERS];      // b_l offset in theta
  int64_t offT[GN_MAX_LAYERS];      // W_l^T offset in the transposed copy (in x out)
  int maxw;                         // widest layer (including input / output)
  int64_t P;                        // parameter count
  int fourier;                      // 1: layer 0 is linear (no activation) and layer 1 the fixed
                                    // Fourier map [cos(B x), sin(B x)] (not in theta; its rows
                                    // are [B; B], its transposed copy sits at offT[1] in wt)
  int exp_out;                      // 1: the outputs are exp of the last layer (else linear)
};

// Arguments of one jet-kernel launch (one point kind).
struct JetArgs {
  NetDesc net;
  int eq;
  int kind;
  int mode;
  const double* theta;   // [P]
  const double* wt;      // transposed weights
  double lam;
  const double* lamp;    // device copy of lambda (null: use lam); graph-captured steps read it here
  int64_t n;             // points of this kind
  const double* y;       // SoA [d][ystride]
  int64_t ystride;
  const double* rho;     // interior weights (may be null)
  double wscale;         // row weight factor (see jet.cu)
  double c_norm;         // normalisation target (KIND_NORM)
  int nfield, nderiv;    // KIND_NORM / KIND_INF: the constrained field, and d/dy1 (NORM only)
  int rsign;             // KIND_RELU: +1 an upper bound (c_norm holds b), -1 a lower bound
  int64_t row0;          // row of point 0, first equation
  double* r;             // r~ output (may be null)
  double* J;             // Jacobian output (MODE_JACOBIAN)
  int64_t ldJ;
  int64_t jrow_lo, jrow_hi;  // rows written are [jrow_lo, jrow_hi), at J + (row - jrow_lo) * ldJ
  double* gpart;         // MODE_GRADIENT: per-warp partial gradients [total warps][ldg]
  int64_t ldg;
  const double* seed;    // MODE_GRADIENT: row seeds (null: seed = r~ itself)
  const double* ug;      // CCF: sum_j K_ij g_j per interior point
  const double* dcoef;   // CCF: diagonal coefficient D_i per interior point
  double* sU;            // CCF out: w_i dR/dU per interior point (times the seed in gradient mode)
  int* flag;             // bit 0: non-finite residual seen
  int lam_frozen;        // lambda held fixed: its Jacobian column and gradient entry are zero
  // stage 2 of multi-stage training: fields Phi_1 + eps Phi_2 with Phi_1's jets precomputed
  // per point (null: single stage).  Interior/wall/norm: base_ld values per point (the probe
  // layout); CCF nodes: g_1 per node.
  const double* base;
  int64_t base_ld;
  double eps;
  const double* fW;      // Fourier layer rows [B; B] (2m' x m, row-major) when net.fourier
};

struct Workspace;
struct GraphState;     // CUDA graphs of the device-resident step (graph.cu)

}  // namespace gn

struct gn_handle {
  gn_problem p;
  int dev;
  cudaStream_t st;
  int eq, d, nf, ne;
  gn::NetDesc net;
  int64_t P, Pp;          // P and P+1
  int64_t n_rows;
  int64_t ldJ;            // leading dimension of the internal J~ (>= P+1, multiple of 16)
  int64_t jrows;          // rows of the internal J~ block buffer
  int precision, n_slices;
  // device workspace
  double* wt;             // transposed weights [P]
  double* theta_t;        // trial parameters [P]
  double* r;              // r~ [n_rows]
  double* J;              // J~ row block [jrows x ldJ]
  double* G;              // Gram [Pp x Pp] row-major, symmetric after mirroring
  double* A;              // factor workspace [Pp x Pp]
  double* Linv;           // inverses of the diagonal blocks [nblk x 64 x 64]
  double* g;              // gradient [Pp]
  double* delta;          // step [Pp]
  double* vtmp;           // scratch [64 x (max(Pp, n_rows) + 16)]
  double* red;            // reduction partials
  int* flag;              // device status word
  double* hpin;           // pinned host scalars
  double* gpart;          // per-warp gradient partials
  int64_t gpart_warps;
  // CCF Hilbert operator (folded on the antisymmetric node pairs)
  int M, Mh;
  double* kf;             // [n_pts x Mh]
  double* dcoef;          // [n_pts]
  double* snode;          // [Mh] positive node coordinates
  double* gnode;          // [Mh] g at the nodes
  double* Jg;             // [Mh x ldJ] Jacobian of g at the nodes (last column d/d lambda)
  double* ug;             // [n_pts]
  double* sU;             // [n_pts]
  double* tnode;          // [Mh] gradient-mode node seeds
  // split-precision Gram workspace (allocated on first use)
  void* split_ws;
  size_t split_ws_bytes;
  void* tmaps;            // host copies of TMA descriptors
  // EMA rank-1 optimiser scratch: u [Pp], J~ Delta [rows], J~ v [rows] (allocated on first use)
  double* ema_ws = nullptr;
  int64_t ema_len = 0;
  // streams of the split factorisation's look-ahead (created on first use)
  cudaStream_t st_hi = nullptr;   // critical path (highest priority)
  cudaStream_t st_lo = nullptr;   // deferred bulk updates (middle priority)
  cudaStream_t st_g = nullptr;    // Gram chunks of the pipelined step (lowest priority)
  // side stream of the wall and normalisation passes (residual and Jacobian modes), with the
  // events that fork it from and join it to the handle's stream
  cudaStream_t st_aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // the split factorisation's own workspace (U, strip operands, diagonal inverses), apart from
  // split_ws so that it can run while the Gram still reads its operand
  void* chol_ws = nullptr;
  size_t chol_ws_bytes = 0;
  // pipelined step: the Gram runs as column-major chunks of at most pipe_tiles 128 x 128 tiles
  // beside the factorisation (0, the default: off, Gram then factorisation; -1: chosen from
  // the SM count)
  int pipe_tiles = 0;
  // graph-captured step (created on first use of gn_step_graph or by a batch capture)
  gn::GraphState* gs = nullptr;
  int capturing = 0;              // a stream capture is in progress: no workspace may grow
  int lam_frozen = 0;             // lambda held fixed (funnel inference trains at fixed lambda)
  int gram_ksplit = 0;            // split-K factor of the split Gram (0: autotuned per shape)
  int gram_tile = 0;              // output tile width of the split Gram, 128 or 64 (0: autotuned)
  // stage 2 of multi-stage training (gn_set_stage1): the stage-1 field jets at every point
  int staged = 0;
  double stage_eps = 1.0;
  int64_t base_ld = 0;
  double* base_int = nullptr;     // [n_pts][base_ld]
  double* base_wall = nullptr;    // [n_bnd][base_ld]
  double* base_norm = nullptr;    // [base_ld]
  double* base_inf = nullptr;     // [n_inf][base_ld]
  double* base_relu = nullptr;    // [n_relu][base_ld]
  double* base_node = nullptr;    // [Mh] (CCF)
  // CCF derivative-loss batches (index 0: d1, 1: d2): series of the folded Hilbert rows and of
  // D in the collocation point, the K part's coefficients at the node values, the row seeds
  double* kd[2] = {nullptr, nullptr};    // [order_y + 1][n_d][Mh]
  double* dd[2] = {nullptr, nullptr};    // [order_y + 1][n_d]
  double* ugd[2] = {nullptr, nullptr};   // [order_y + 1][n_d]
  double* sUd[2] = {nullptr, nullptr};   // [ord + 1][n_d]
  double* fourierW = nullptr;     // Fourier layer rows [B; B] (2m' x m), when the network has one
};

namespace gn {

// One evaluation pass over all point kinds (gn_api.cu).
struct Pass {
  int mode;
  double* r;        // r~ destination (may be null)
  double* J;        // Jacobian block destination
  int64_t ldJ, jlo, jhi;
  const double* seed;
  const double* lamp = nullptr;   // device lambda (null: the host value passed to run_pass)
  bool unweighted = false;        // interior rows carry R itself (no loss weights)
};
int run_pass(gn_handle* h, const double* theta, double lam, const Pass& ps, double* grad);
// 1/2 |r|^2 reduction: the sum of squares lands in red[256 + slot] (device)
int loss_of(gn_handle* h, const double* r, int slot);
// max |R_k| over the interior points of rows r (unweighted) into red[kMaxResSlot] (device)
constexpr int kMaxResSlot = 270;
int max_res_of(gn_handle* h, const double* r);
int gram_into(gn_handle* h, const double* J, int64_t ld, int64_t nrows, const double* r, double* G, double* g,
              int precision, int accumulate);
// grow the split workspace to what every split contraction of a step needs, and create the
// factorisation's streams, so that a captured step allocates nothing
int prepare_for_capture(gn_handle* h);
size_t chol_split_ws_bytes(int64_t n, int S);
// split-K factor and tile width the Gram autotuner recorded for this shape (0: not tuned yet)
int gram_split_choice(int S, int64_t Pp, int64_t nrows);
int gram_tile_choice(int S, int64_t Pp, int64_t nrows);
cudaError_t ensure_chol_streams(gn_handle* h);
void graph_release(gn_handle* h);

// ---- launchers (host functions implemented in the .cu files) -----------
cudaError_t launch_transpose_weights(const NetDesc& net, const double* theta, double* wt, cudaStream_t st);
cudaError_t launch_jet(const JetArgs& a, cudaStream_t st, int64_t* warps_used);
// derivative-loss rows of order ord (1: d1, 2: d2) at the a.n points (djet.cu); a.row0 is the
// first row, a.wscale sqrt(2 c_d / (N_d N_E d^ord)).  CCF: a.ug / a.dcoef hold the K part's
// and D's Taylor coefficients in y ([m][n], m <= order_y), a.sU receives d row / d U_m ([m][n],
// m <= ord; times the combined seed in gradient mode)
cudaError_t launch_djet(const JetArgs& a, int ord, cudaStream_t st, int64_t* warps_used);
// degree in y of the field series of the derivative rows of order ord in d dimensions
inline int djet_order_y(int d, int ord) { return (d == 1 ? 1 : 2) + ord; }
int jet_gpart_warps(const NetDesc& net, int d, int nf, int64_t n_max);
cudaError_t launch_gpart_reduce(const double* gpart, int64_t warps, int64_t ldg, int64_t n,
                                double* out, int accumulate, cudaStream_t st);

// FP64 GEMM: C(m x n) = alpha * sum_k A(m,k) B(k,n) + beta * C, optional row scale.
// a_kcontig: A(m,k) = A[m*lda + k] (else A[k*lda + m]); b_kcontig: B(k,n) = B[n*ldb + k]
// (else B[k*ldb + n]).  lower: only tiles with row tile >= col tile are computed.
// rowscale (may be null): C[m][n] = beta C + rowscale[m] * alpha * acc.
cudaError_t dgemm(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                  bool a_kcontig, const double* B, int64_t ldb, bool b_kcontig, double beta, double* C,
                  int64_t ldc, bool lower, const double* rowscale, cudaStream_t st);

// Vector helpers (deterministic reductions).
cudaError_t dot_partial(const double* x, const double* y, int64_t n, double* red, cudaStream_t st);
// EMA rank-1 optimiser: G = u u^T (first) or beta G + (1 - beta) u u^T; the two-term update
cudaError_t ema_rank1(double* G, int64_t n, int64_t ld, const double* u, double beta, int first, cudaStream_t st);
cudaError_t ema_update(const double* theta, const double* delta, double* v, double alpha, double mu, int64_t P,
                       int64_t n, double* theta_t, cudaStream_t st);
cudaError_t sumsq_and_flag(const double* x, int64_t n, double* red, cudaStream_t st);
cudaError_t finish_sum(double* red, double* out_dev, cudaStream_t st);
cudaError_t axpy_trial(const double* theta, const double* delta, double alpha, int64_t P, double* out,
                       cudaStream_t st);
// y[n] = beta*y + A^T x, A is m x n row-major; part: scratch of kGemvChunks * n doubles
constexpr int kGemvChunks = 64;
cudaError_t dgemv_t_scratch(const double* A, int64_t lda, int64_t m, int64_t n, const double* x, double* y,
                            double beta, double* part, cudaStream_t st);
cudaError_t dgemv_n(const double* A, int64_t lda, int64_t m, int64_t n, const double* x, double* y,
                    double beta, cudaStream_t st);   // y[m] = beta*y + A x
cudaError_t mirror_lower(double* G, int64_t n, int64_t ld, cudaStream_t st);
// A = G + gamma I on the lower triangle's columns [c0, c1) (gamma: device scalar)
cudaError_t add_diag_band(const double* G, double* A, int64_t n, int64_t ld, int64_t c0, int64_t c1,
                          const double* gamma, cudaStream_t st);
// y with x . y = x^T G x from G's lower triangle: y_i = G_ii x_i + 2 sum_{j<i} G_ij x_j
cudaError_t quad_lower(const double* G, int64_t n, int64_t ld, const double* x, double* y, cudaStream_t st);
// A = G + gamma I on the lower triangle (gamma_dev, when given, is read on the device instead)
cudaError_t copy_add_diag(const double* G, double* A, int64_t n, int64_t ld, double gamma, const double* gamma_dev,
                          cudaStream_t st);
cudaError_t max_abs_rows(const double* r, int64_t n, int stride_valid, double* red, cudaStream_t st);
cudaError_t finish_max(double* red, double* out_dev, cudaStream_t st);
// max |R_k| over the interior rows r_i = w sqrt(rho_i) R_k (rho null: 1) into *out_dev
cudaError_t max_abs_unweighted(const double* r, int64_t n_pts, int ne, const double* rho, double w, double* red,
                               double* out_dev, cudaStream_t st);

// CCF Hilbert operator construction and contractions.
cudaError_t hilbert_build(const double* y, int64_t n, int M, double* kf, double* dcoef, double* snode,
                          cudaStream_t st);
// Taylor coefficients m = 0..order in the collocation point x of the folded K row and of D:
// kd[m][i][j'] (n x M/2 each), dd[m][i]
cudaError_t hilbert_series_build(const double* y, int64_t n, int M, int order, double* kd, double* dd,
                                 cudaStream_t st);

// Cholesky (FP64, blocked, lower, in place on A row-major) and solves.
constexpr int kCholNB = 64;
constexpr int64_t kCholStrip = 4 * kCholNB;   // columns per strip of the split factorisation
cudaError_t cholesky_factor(double* A, int64_t n, int64_t lda, double* Linv, int* flag, cudaStream_t st);
cudaError_t cholesky_solve(const double* A, int64_t n, int64_t lda, const double* Linv, const double* b,
                           double* x, double* tmp, cudaStream_t st);   // tmp: 2n doubles
// L^T x = y only (the forward half already done, e.g. inside cholesky_factor_split); tmp: n doubles
cudaError_t cholesky_solve_backward(const double* A, int64_t n, int64_t lda, const double* Linv, const double* y,
                                    double* x, double* tmp, cudaStream_t st);

// Split-precision (Ozaki, BF16 slices on tcgen05) GEMM C op= A B^T (ozaki.cu).
// An operand holds S BF16 slices [S][npad][kpad] (K-major) and one power-of-two
// exponent per row (npad rows, padded with zeros).
constexpr int kOzMaxSlices = 6;
struct OzOperand {
  void* slices;          // __nv_bfloat16 [S][npad][kpad]
  int* e;                // [npad]
  int64_t npad, kpad;    // npad is also the row stride between slices
  int64_t kuse = 0;      // contraction length actually used (a multiple of 32; 0: kpad)
  int64_t map_rows = 0;  // rows addressable from `slices` in the 2D slice view (0: S npad)
  // chunked exponents: echunk > 0 gives every row one exponent per echunk contraction
  // columns, chunk c's at e[c * estride + row] (echunk a multiple of 32, at most 128)
  int echunk = 0;
  int64_t estride = 0;
};
// rows [row_off, ...) of op as an operand of its own (same slice stride; row_off % 8 == 0)
OzOperand oz_operand_rows(const OzOperand& op, int S, int64_t row_off);
// Slices of one value x of an operand row with exponent e (2^e > max |row|): the
// integer round(x 2^{8S-e}) written in balanced base-256 digits a_0 .. a_{S-1}
// (a_0 carries the sign and the rest lie in [-128, 128)); slice q holds
// a_q 2^{-8(q+1)}, exact in BF16.  out[q * stride] receives slice q.
// round(x 2^n) to the nearest integer, ties to even (what llrint(ldexp(x, n)) gives), by
// integer operations on the bits: GB300 runs the FP64 scaling and the FP64 -> int64
// conversion on its narrow FP64 pipe, which made the slicing passes FP64-bound.  Results that
// leave the range the split uses (|x 2^n| >= 2^62) and non-finite x take the FP64 path.
__device__ __forceinline__ long long scaled_rint(double x, int n) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0x7ff) return llrint(ldexp(x, n));
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  int ee = ex;
  if (ex != 0) m |= 1ull << 52;   // normal: the implicit bit
  else ee = 1;                    // subnormal
  const int sh = ee - 1075 + n;   // x 2^n = +-m 2^sh
  unsigned long long q;
  if (sh >= 0) {
    if (sh > 9) return llrint(ldexp(x, n));
    q = m << sh;
  } else if (-sh >= 64) {
    q = 0;                        // m < 2^53 <= 2^(-sh - 1): rounds to zero
  } else {
    const int r = -sh;
    q = m >> r;
    const unsigned long long rem = m & ((1ull << r) - 1), half = 1ull << (r - 1);
    if (rem > half || (rem == half && (q & 1))) q++;
  }
  return (b >> 63) ? -(long long)q : (long long)q;
}
template <int S>
__device__ __forceinline__ void oz_digits(double x, int e, __nv_bfloat16* out, int64_t stride) {
  long long v = scaled_rint(x, 8 * S - e);
  int a[S];
#pragma unroll
  for (int q = S - 1; q >= 1; q--) {
    const long long d = (v + 128) >> 8;
    a[q] = (int)(v - (d << 8));
    v = d;
  }
  a[0] = (int)v;
#pragma unroll
  for (int q = 0; q < S; q++) out[q * stride] = __float2bfloat16_rn(ldexpf((float)a[q], -8 * (q + 1)));
}
size_t oz_operand_bytes(int S, int64_t n, int64_t k);
OzOperand oz_operand_at(void* base, int S, int64_t n, int64_t k);
// X is K x n row-major (operand row j = column j of X); part: 64 * npad doubles of scratch
int oz_prepare_cols(int S, const double* X, int64_t ld, int64_t k, int64_t n, const OzOperand& op, double* part,
                    cudaStream_t st);
// X is n x K row-major (operand row j = row j of X)
int oz_prepare_rows(int S, const double* X, int64_t ld, int64_t n, int64_t k, const OzOperand& op,
                    cudaStream_t st);
// C (M x N, ldc) op= A B^T; sym: only tiles with row tile >= column tile (A must equal B);
// mode 0: C = v, 1: C += rowscale[i] v (rowscale may be null), 2: C -= v.  flag: bit 1 on timeout.
// ksplit > 1 (modes 0-2, single exponents only): the contraction is cut into ksplit parts
// over that many more CTAs, whose partial tiles (part: tiles * ksplit * 128 * 128 float2)
// are summed by a second launch.
// range (sym only): just the tiles [tile0, tile0 + ntiles) of the lower triangle, numbered row by
// row or, with colmajor, column by column (the first c mt - c (c - 1) / 2 tiles are tile columns
// 0 .. c - 1, mt = ceil(M / 128)); ntiles < 0: every tile.
struct OzRange {
  int64_t tile0 = 0, ntiles = -1;
  int colmajor = 0;
};
// tile_n: output tile columns, 128 (the default) or 64 (twice the tiles of a narrow or small C)
int oz_gemm(int S, bool sym, const OzOperand& A, const OzOperand& B, int64_t M, int64_t N, double* C, int64_t ldc,
            int mode, const double* rowscale, int* flag, cudaStream_t st, int ksplit = 1, void* part = nullptr,
            const OzRange& range = OzRange(), int tile_n = 128);
// Gram through oz_gemm (lower tiles); returns GN_ERR_* codes.
int split_gram(gn_handle* h, const double* J, int64_t ld, int64_t nrows, double* G, int accumulate);
// Tiles per chunk of the pipelined Gram for this handle's step, 0 when the step does not
// pipeline (another precision, several row blocks, split-K, a small G or pipe_tiles == 0).
int64_t pipeline_chunk_tiles(gn_handle* h);
// The pipelined Gram: J~'s operand on st, then sg forked from st and, on sg, the lower tiles of
// G column by column in launches of at most `chunk` tiles; after each launch, the 256-column
// strips it finished are copied into A = G + gamma I (lower triangle; gamma a device scalar) and
// gate[t] is set to an event recorded after their copy (one per strip).  Last, G's upper
// triangle is mirrored on sg.  Events are created into `events`; the caller destroys them once
// the work is captured or done, and joins sg back.
int split_gram_pipelined(gn_handle* h, const double* J, int64_t ld, int64_t nrows, double* G, double* A,
                         const double* gamma, int64_t chunk, cudaStream_t st, cudaStream_t sg,
                         std::vector<cudaEvent_t>& events, std::vector<cudaEvent_t>& gate);
// grow the handle's split workspace to at least `need` bytes
int ensure_split_ws(gn_handle* h, size_t need);
// blocked Cholesky whose trailing updates run through oz_gemm
// (with b: also the forward substitution L y = b, w being n doubles of work space)
// gate (may be null): one event per 256-column strip (null entries: none); the strip's chain
// waits for its event before it reads the strip's columns of A.
cudaError_t cholesky_factor_split(gn_handle* h, double* A, int64_t n, int64_t lda, double* Linv, int* flag, int S,
                                  const double* b, double* y, double* w, int* rc_out,
                                  const cudaEvent_t* gate = nullptr);
// the factorisation's workspace, grown to `need` bytes (never inside a capture)
int ensure_chol_ws(gn_handle* h, size_t need);

}  // namespace gn
