/*
 * gn.h -- C ABI of the GB300 Gauss-Newton profile-fit library (libgn.so).
 *
 * The library evaluates, on one GPU, the hot path of the method of
 * "Discovery of Unstable Singularities" (arXiv 2509.14185): a small tanh MLP
 * models a self-similar blow-up profile (Methods, Eq. self-similar and Eq.
 * ansatz_vorticity), each collocation point contributes the residuals R_k of
 * the static self-similar equations (Eq. self-similar-static, "Training
 * Loss"), and one damped Gauss-Newton step (Methods, "Second-order
 * Optimizer") updates the network parameters theta and the blow-up rate
 * lambda together (lambda as a trainable unknown, "Identifying Admissible
 * lambda Values", item 1).
 *
 * Conventions used by every call:
 *   - All floating point is IEEE binary64 ("FP64") unless a call says otherwise.
 *   - "device" pointers are CUDA global-memory addresses on the GPU that was
 *     current when gn_init ran; "host" pointers are ordinary CPU memory.
 *   - Every call is asynchronous with respect to the host only where stated;
 *     calls that return scalars to the host synchronise the handle's stream.
 *   - Functions never abort and never print.  They return GN_OK (0), a
 *     positive warning, or a negative GN_ERR_* code; gn_error_string maps a
 *     code to a static message.
 *   - Parameters: theta holds, for each linear layer l in order, the weight
 *     matrix W_l (out_l x in_l, row-major) followed by the bias b_l (out_l).
 *     P = sum_l (in_l*out_l + out_l).  lambda is passed separately; the
 *     Jacobian has P' = P + 1 columns and column P is d/d lambda.
 *   - Rows: r~ has n_rows = n_pts * N_E + n_d1 * N_E * d + n_d2 * N_E * d^2
 *     + n_bnd + n_inf + n_relu + 1 entries, in the order (interior point i,
 *     equation k) at row i*N_E + k, then the d1 rows (point, k, i), the d2
 *     rows (point, k, i, j), the wall rows, the decay rows, the bound rows,
 *     and the normalisation row last.  Rows are weighted so that
 *     h = 1/2 |r~|^2 = (1/(n_pts N_E)) sum_i rho_i sum_k R_k(y_i)^2
 *                      + c_d1 L_d1 + c_d2 L_d2
 *                      + (c_bnd/n_bnd) sum_b Psi(y_b)^2
 *                      + c_inf sum Phi_A0(y)^2 + c_relu sum relu(...)^2
 *                      + c_norm_w (Phi_A0(y_norm) - c_norm)^2,
 *     i.e. the paper's equation loss plus its data loss ("Training Loss").
 *     Then grad h = J~^T r~ and the Gauss-Newton matrix is G = J~^T J~.
 */
#ifndef GN_H_
#define GN_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define GN_OK                 0
#define GN_WARN_NO_DECREASE   1   /* line search found no decrease: theta, lambda kept, damping *= 10 */
#define GN_ERR_INVALID       -1   /* bad argument (null pointer, size, unsupported shape) */
#define GN_ERR_CUDA          -2   /* a CUDA runtime call failed */
#define GN_ERR_OOM           -3   /* device allocation failed */
#define GN_ERR_NONFINITE     -4   /* a residual or loss was NaN or infinite */
#define GN_ERR_NOT_SPD       -5   /* G + gamma I not positive definite after 5 damping escalations */
#define GN_ERR_TIMEOUT       -6   /* a bounded device-side wait gave up */
#define GN_ERR_UNSUPPORTED   -7   /* requested precision/path not available on this device */
#define GN_ERR_TOO_LARGE     -8   /* size exceeds the fixed scratch of gn_jtr_noalloc (16384 columns) */
#define GN_ERR_IO            -9   /* a checkpoint file could not be written or read */
#define GN_ERR_MISMATCH     -10   /* a checkpoint belongs to another equation or architecture */

/* ---- problem description ----------------------------------------------- */
/* Equations (Results and Methods; residual operators as derived from the
 * paper's ansatz, see R_k below). */
enum gn_equation {
  GN_BURGERS = 0,     /* 1D Burgers, the paper's worked example (research flowchart figure):
                         R = -lambda U + ((1+lambda) y + U) U'                           */
  GN_CCF = 1,         /* 1D Cordoba-Cordoba-Fontelos, theta_t + (H theta) theta_x = 0:
                         R = -lambda Theta + ((1+lambda) y + H Theta) Theta'              */
  GN_IPM = 2,         /* 2D incompressible porous media with wall y2 = 0, fields (P, Psi):
                         R1 = -lambda P + V.grad P, R2 = Laplace Psi - d1 P               */
  GN_BOUSSINESQ = 3   /* 2D Boussinesq with wall y2 = 0, fields (Omega, Theta, Psi):
                         R1 = Omega + V.grad Omega - d1 Theta,
                         R2 = (1-lambda) Theta + V.grad Theta, R3 = Laplace Psi + Omega
                         (V = (1+lambda) y + U, U = (d2 Psi, -d1 Psi))                    */
};

/* Precision of the Gram product G = J~^T J~ (Methods, "Second-order Optimizer";
 * everything else is always FP64). */
enum gn_precision {
  GN_PREC_FP64 = 0,        /* native FP64 (DFMA) Gram */
  GN_PREC_SPLIT_BF16 = 1,  /* Ozaki split: each FP64 column of J~ scaled by a power of two and
                              split into n_slices BF16 slices; slice products on the tcgen05
                              tensor cores with exactly representable FP32 partial sums,
                              combined in double-FP32 and returned as FP64 */
  GN_PREC_SPLIT_ALL = 2    /* as GN_PREC_SPLIT_BF16, and the other two dense contractions too:
                              the CCF Hilbert contraction J_U = K J_g and the trailing updates
                              of the blocked Cholesky factorisation (accumulated in double-FP32;
                              diagonal blocks and panels in double-float arithmetic, ~48 bits;
                              triangular solves FP64; backward error ~2e-13).  Entrywise error of
                              each split product, in units of 2^(e_i+e_j) with |x| < 1 the
                              power-of-two scaled operands and K the contraction length:
                              2^(-8S-1)(|x_i|_1+|x_j|_1) + K 2^(-16S-2) + K S(S-1) 2^(-8S-3)
                              + [S>=4] K_pad K S 2^(-52)                                    */
};

#define GN_MAX_LAYERS 8

typedef struct gn_problem {
  int equation;              /* enum gn_equation */
  int n_layers;              /* number of linear layers L (hidden layers + output layer), 1..GN_MAX_LAYERS */
  int widths[GN_MAX_LAYERS + 1]; /* widths[0] = d (1 or 2), widths[L] = number of fields
                                   (1 Burgers/CCF, 2 IPM, 3 Boussinesq); hidden widths 1..256 */
  int64_t n_pts;             /* interior collocation points (>= 0) */
  const double* y;           /* device, SoA [d][n_pts]: y[k*n_pts + i] is coordinate k of point i.
                                Borrowed: must stay valid until gn_destroy. */
  const double* rho;         /* device [n_pts] per-point loss weights, or NULL for all ones. Borrowed. */
  int64_t n_bnd;             /* wall points (2D problems only; must be 0 for 1D) */
  const double* y_bnd;       /* device, SoA [2][n_bnd], points on the wall y2 = 0. Borrowed. */
  double c_bnd;              /* weight of the wall loss (mean over wall points); 1.0 by default */
  double y_norm[2];          /* normalisation point (Methods, "Training Loss", data loss) */
  double c_norm;             /* target value C_norm */
  double c_norm_w;           /* weight c_norm of the normalisation row */
  int hilbert_m;             /* CCF only: nodes M of the discrete Hilbert operator (even, 8..16384) */
  int precision;             /* enum gn_precision used by gn_step for the Gram */
  int n_slices;              /* split precision only: BF16 slices per FP64 value (1..6) */
  int fourier_m;             /* 0: tanh MLP.  > 0: Fourier-feature network (Methods, "Multi-stage
                                Training", item 2): layer 0 is the linear input layer (no
                                activation, widths[1] = m), layer 1 the fixed map
                                x -> [cos(B x), sin(B x)] (widths[2] = 2 fourier_m, no parameters,
                                not in theta), then tanh layers and the linear output layer;
                                n_layers >= 3 */
  const double* fourier_B;   /* host [fourier_m x widths[1]] row-major, B ~ N(0, sigma^2) drawn by
                                the caller; copied by gn_init */
  int64_t n_inf;             /* decay points Y_inf of the data loss (Methods, "Training Loss"): rows
                                sqrt(2 c_inf) Phi_A0(y), the value of the normalised field (field 0),
                                placed after the wall rows and before the normalisation row; 0: none */
  const double* y_inf;       /* device, SoA [d][n_inf]. Borrowed: must stay valid until gn_destroy. */
  double c_inf;              /* weight c_inf of the decay rows (the loss gains c_inf sum Phi_A0(y)^2) */
  int norm_kind;             /* the normalisation constraint (Methods, "Training Loss": on a field's
                                value or derivative): 0 the equation's own (value of field 0;
                                Boussinesq d Omega / d y1), 1 the value of field norm_field,
                                2 its d/dy1.  The decay rows take the value of the same field. */
  int norm_field;            /* field A0 for norm_kind 1 and 2 (0 .. fields - 1) */
  int output_map;            /* last activation of the network (Methods, "Solution Modeling":
                                exponential or exponential-adjacent): 0 linear (default), 1 exp,
                                NN_A = exp(W_L h + b_L); a stage-1 network (gn_set_stage1) uses
                                the same map */
  int64_t row_block;         /* rows per Jacobian block of a step (0: automatic, the whole J~ when
                                it fits 32 GiB, else the largest block that does); smaller blocks
                                stream J~ through a smaller buffer, the Gram accumulating over them */
  int64_t n_relu;            /* bound points of the data loss (Methods, "Training Loss": a constraint
                                acted on by a relu before squaring): rows sqrt(2 c_relu)
                                relu(s (Phi_A0(y) - relu_bound)) after the decay rows; 0: none */
  const double* y_relu;      /* device, SoA [d][n_relu]. Borrowed: must stay valid until gn_destroy. */
  double c_relu;             /* weight of the bound rows */
  double relu_bound;         /* the bound b on the constrained field */
  int relu_sign;             /* s: >= 0 an upper bound (Phi_A0 <= b), < 0 a lower bound (Phi_A0 >= b) */
  int64_t n_d1;              /* points of the d1 derivative loss (Methods, "Training Loss": the
                                residuals' first y-derivatives, its own batch Y_1): rows
                                sqrt(2 c_d1 rho / (n_d1 N_E d)) d_{y_i} R_k(y), point-major, then k,
                                then i, placed after the interior rows; 0: none.  For CCF the
                                velocity is the discrete Hilbert operator differentiated in the
                                collocation point (node values fixed).  Not with fourier_m > 0,
                                output_map = 1 or a second stage (GN_ERR_UNSUPPORTED). */
  const double* y_d1;        /* device, SoA [d][n_d1]. Borrowed: must stay valid until gn_destroy. */
  const double* rho_d1;      /* device [n_d1] point weights rho, or NULL for all ones. Borrowed. */
  double c_d1;               /* coefficient c_d1 of the d1 loss */
  int64_t n_d2;              /* points of the d2 derivative loss: rows sqrt(2 c_d2 rho / (n_d2 N_E d^2))
                                d_{y_i} d_{y_j} R_k(y) for every ordered pair (i, j) (the mixed pair
                                twice in 2D, as the paper's double sum counts it), after the d1 rows */
  const double* y_d2;        /* device, SoA [d][n_d2]. Borrowed. */
  const double* rho_d2;      /* device [n_d2] point weights, or NULL for all ones. Borrowed. */
  double c_d2;               /* coefficient c_d2 of the d2 loss */
} gn_problem;

/* Normalisation row (data loss) per equation, fixed by the library:
 *   Burgers U(y_norm), CCF Theta(y_norm), IPM P(y_norm), Boussinesq d Omega/d y1 (y_norm). */

typedef struct gn_step_info {
  double loss_before;        /* h(theta, lambda) */
  double loss_after;         /* h at the accepted point (== loss_before if none) */
  double alpha;              /* accepted step length (0 if none) */
  double rho;                /* Levenberg-Marquardt ratio actual/predicted decrease */
  double gamma_used;         /* damping that the accepted factorisation used */
  int chol_retries;          /* damping escalations needed to factorise */
  int n_trials;              /* residual-only line-search evaluations */
  int status;                /* same value as the return code */
  double ms_phase[8];        /* device time per phase: jacobian, gram, gradient, factor,
                                solve, line search, total, unused */
  double momentum;           /* gn_step_ema: the closed-form momentum coefficient mu (0 in gn_step) */
  double max_abs_res;        /* gn_step and gn_step_graph: max |R_k| over the interior points and
                                equations at the step's starting point (theta, lambda), unweighted
                                (Methods, "Validation Metrics", max d0 residual on the collocation
                                points), from the rows the step evaluates anyway; the accepted
                                point's value is the next step's.  NaN if a row was not finite. */
} gn_step_info;

typedef struct gn_handle gn_handle;

/* ---- lifecycle ------------------------------------------------------------ */

/* Create a handle for one profile fit.  Copies *p (the point arrays stay
 * borrowed), allocates all device workspace (J~, G, factor, vectors, the CCF
 * Hilbert matrix) on the current device, and binds the handle to
 * cuda_stream (a cudaStream_t; NULL = legacy default stream).
 * Cites: problem statement in Methods ("Self-similar Solutions", "Solution
 * Modeling", "Training Loss").  Errors: GN_ERR_INVALID, GN_ERR_OOM, GN_ERR_CUDA. */
int gn_init(const gn_problem* p, void* cuda_stream, gn_handle** out);

/* Release all device workspace owned by the handle.  Safe on NULL. */
int gn_destroy(gn_handle* h);

/* P (network parameters, excluding lambda) and the number of rows of r~. */
int gn_param_count(const gn_handle* h, int64_t* P);
int gn_row_count(const gn_handle* h, int64_t* n_rows);

/* Change the Gram precision used by gn_step and gn_gram. */
int gn_set_precision(gn_handle* h, int precision, int n_slices);

/* Split-K factor of the split-precision Gram (the contraction over rows cut into ksplit
 * parts over ksplit times more CTAs, partial tiles summed in a fixed order by a second
 * launch).  ksplit = 0 (default): autotuned: on the first split Gram of a shape (slices,
 * column tiles, contraction chunks) in the process, every candidate (1 and the splits that
 * keep the launch within four waves of the 152 SMs and at least 256 rows per part) is
 * timed with CUDA events on the handle's stream and the fastest kept for every handle of
 * that shape; the tuning launch synchronises the stream.  ksplit = 1..8 forces a factor.
 * The split changes only the order of the final FP64 additions.  GN_ERR_INVALID otherwise.
 * gn_gram_split_choice reports the factor a Gram over nrows rows uses (0: not tuned yet). */
int gn_set_gram_split(gn_handle* h, int ksplit);
int gn_gram_split_choice(const gn_handle* h, int64_t nrows, int* ksplit);

/* Output tile shape of the split-precision Gram (the batched sweep's configuration asks for Gram
 * tile shapes picked by an autotuner): 128 x 128 tiles, or 128 x 64 tiles (twice the CTAs, each
 * with half the B operand and half the tensor memory; more parallelism for a small P').
 * tile_n = 0 (default): autotuned together with the split-K factor on the first split Gram of a
 * shape, over every (tile width, split-K) candidate, the default kept unless another is at least
 * 3 % faster; tile_n = 128 or 64 forces one (with a forced width or split-K the other is not
 * tuned).  The tile shape changes only which CTA computes an entry, not its arithmetic: results
 * are bit for bit the same.  The pipelined step (gn_set_pipeline) uses 128-column tiles only.
 * gn_gram_tile_choice reports the width a Gram over nrows rows uses (0: not tuned yet).
 * GN_ERR_INVALID for other values. */
int gn_set_gram_tile(gn_handle* h, int tile_n);
int gn_gram_tile_choice(const gn_handle* h, int64_t nrows, int* tile_n);

/* Pipelined Gram and factorisation in gn_step_graph (precision GN_PREC_SPLIT_ALL, one row
 * block, split-K factor 1).  The lower tiles of G = J~^T J~ are computed column by column in
 * chunks of at most `tiles` 128 x 128 tiles (one launch each, on a stream of the lowest
 * priority); the damped copy A = G + gamma I of each finished band of 256 columns is made at
 * once, and the factorisation's chain (highest priority) starts each 256-column strip as soon as
 * its band is in A, so the latency-bound factorisation runs beside the tensor-bound Gram on the
 * SMs the chunks leave free.  The arithmetic is unchanged: results equal the unpipelined step
 * bit for bit.  tiles = 0 (the default) keeps the unpipelined order (Gram, then factorisation);
 * -1 picks 7/8 of the SM count; a change takes effect at the next capture.  On GB300 the
 * factorisation's wide kernels (panel solves, trailing updates) slow down on the SMs the chunks
 * leave free about as much as the overlap saves, hence off by default.  GN_ERR_INVALID for
 * tiles < -1.  Cites: Methods, "Second-order Optimizer" (the damped normal equations the step
 * solves); the pipelining is this library's scheduling. */
int gn_set_pipeline(gn_handle* h, int tiles);
/* *tiles = tiles per Gram chunk that the next capture of gn_step_graph uses (0: the step does
 * not pipeline: another precision, several row blocks, a split-K Gram, fewer than 4 tile
 * columns, or the pipeline off).  GN_ERR_INVALID for null arguments. */
int gn_pipeline_tiles(gn_handle* h, int64_t* tiles);

/* ---- evaluation --------------------------------------------------------- */

/* r_out[0..n_rows) = r~(theta, lambda); *loss_out (host, may be NULL) = h = |r~|^2/2.
 * theta: device [P].  r_out: device [n_rows], caller-owned (may be NULL when
 * only the loss is wanted).  Synchronises the stream when loss_out != NULL.
 * Returns GN_ERR_NONFINITE if the loss is not finite.
 * Cites: residual factorisation E_k = F_k R_k and the d0 loss (Methods,
 * "Solution Modeling" and "Training Loss"). */
int gn_residual(gn_handle* h, const double* theta, double lambda, double* r_out, double* loss_out);

/* Rows [row0, row0+nrows) of J~ = d r~ / d(theta, lambda) into J_out (device,
 * row-major, leading dimension ld >= P+1; column P is d/d lambda, the total
 * derivative through the coordinates q(y; lambda), the envelopes and the
 * explicit lambda terms).  Caller owns J_out.  Asynchronous.
 * Cites: Gauss-Newton matrix built from Jacobian products (Methods,
 * "Second-order Optimizer"). */
int gn_jacobian(gn_handle* h, const double* theta, double lambda, double* J_out, int64_t ld,
                int64_t row0, int64_t nrows);

/* grad_out[0..P] = J~^T seed without forming J~ (reverse pass through the
 * jets, one per collocation point).  seed: device [n_rows], or NULL for
 * seed = r~ (then grad_out = grad h).  grad_out: device [P+1], caller-owned.
 * Asynchronous.  This is the adjoint that backs torch.autograd. */
int gn_gradient(gn_handle* h, const double* theta, double lambda, const double* seed, double* grad_out);

/* ---- Gauss-Newton pieces -------------------------------------------------- */

/* G_out = J^T J (lower triangle; the strict upper triangle is also written
 * for precision FP64, left untouched for SPLIT) and g_out = J^T r for a
 * caller-given row block.  J: device [nrows x ld] row-major with P+1 used
 * columns; r: device [nrows] (may be NULL, then g_out is not written);
 * G_out: device [(P+1) x (P+1)] row-major; g_out: device [P+1].
 * accumulate != 0 adds into G_out/g_out instead of overwriting (row-block
 * streaming).  precision: enum gn_precision.  Asynchronous. */
int gn_gram(gn_handle* h, const double* J, int64_t ld, int64_t nrows, const double* r,
            double* G_out, double* g_out, int precision, int accumulate);

/* delta_out = (G + gamma I)^{-1} g by a blocked FP64 Cholesky factorisation,
 * escalating gamma *= 10 (at most 5 times) when a pivot is not positive.
 * G: device [(P+1)^2] row-major (lower triangle read, not modified);
 * g, delta_out: device [P+1]; *gamma in/out (host); *retries_out (host, may
 * be NULL).  Synchronises.  Returns GN_ERR_NOT_SPD when all retries fail. */
int gn_damped_solve(gn_handle* h, const double* G, const double* g, double* gamma,
                    double* delta_out, int* retries_out);

/* One damped Gauss-Newton step, in place:
 *   r~, J~ at (theta, lambda); G = J~^T J~ (precision of the handle);
 *   g = J~^T r~; delta = (G + gamma I)^{-1} g; Armijo backtracking on
 *   alpha = 1, 1/2, ... (<= 8 residual-only evaluations, c1 = 1e-4);
 *   theta -= alpha delta[0..P), lambda -= alpha delta[P];
 *   Levenberg-Marquardt update of gamma (x1.5 if rho < 1/4, x2/3 if rho > 3/4).
 * theta: device [P] in/out; lambda, damping: host in/out; info: host (may be NULL).
 * Returns GN_OK, GN_WARN_NO_DECREASE (theta and lambda unchanged, damping
 * x10), GN_ERR_NOT_SPD or GN_ERR_NONFINITE.  Synchronises.
 * Cites: Methods, "Second-order Optimizer" (damped Gauss-Newton update and
 * Levenberg-Marquardt damping); the line-search and LM constants are this
 * library's choice because the paper gives none. */
int gn_step(gn_handle* h, double* theta, double* lambda, double* damping, gn_step_info* info);

/* The step of gn_step with every host decision moved onto the device, captured
 * once as CUDA graphs and replayed: the factorisation check, the Armijo
 * backtracking (eight conditional IF nodes, one residual-only trial each) and
 * the Levenberg-Marquardt update read and write a device-resident state holding
 * lambda and the damping, so one step is one graph launch plus one small copy
 * each way and one synchronisation.  Same arguments, results, constants and
 * return codes as gn_step (a failed factorisation replays the solve part with
 * damping x10, at most 5 times).  The first call for a given theta address (or
 * after gn_set_precision or a change of the lambda setting) captures the
 * graphs: it grows the handle's workspace to its final size and synchronises;
 * make that first call before any stream capture of your own.  The graphs run
 * on a stream of the handle's own, after the work already queued on the
 * handle's stream.  info->ms_phase[6] is the step's device time; the other
 * phases are not timed.  Cites: Methods, "Second-order Optimizer". */
int gn_step_graph(gn_handle* h, double* theta, double* lambda, double* damping, gn_step_info* info);

/* ---- batched fits ---------------------------------------------------------- */
/* Many independent profile fits of uneven size (lambda seeds, widths, depths,
 * point counts), as in the paper's sweeps over lambda and seeds (Methods,
 * "Identifying Admissible lambda Values" and "Validation of lambda").  The
 * fits share nothing; they are dealt round-robin onto n_streams CUDA streams
 * created by the batch, and gn_batch_step drives one damped GN step of every
 * fit with one host worker thread per stream, so their kernels overlap on the
 * GPU.  problems: host array [n_fits] (point arrays borrowed as in gn_init).
 * Errors: as gn_init; on failure nothing is left allocated. */
typedef struct gn_batch gn_batch;
int gn_batch_init(const gn_problem* problems, int n_fits, int n_streams, gn_batch** out);
/* The handle of one fit (owned by the batch; valid until gn_batch_destroy). */
int gn_batch_handle(gn_batch* b, int fit, gn_handle** out);
/* One gn_step of every fit.  thetas: host array of n_fits device pointers;
 * lambdas, dampings: host [n_fits] in/out; infos (host [n_fits], may be NULL);
 * status (host [n_fits], may be NULL) receives each fit's return code.
 * Returns GN_OK or the most negative error code of any fit.  Synchronises. */
int gn_batch_step(gn_batch* b, double* const* thetas, double* lambdas, double* dampings, gn_step_info* infos,
                  int* status);
int gn_batch_destroy(gn_batch* b);

/* Graph mode of a batch: one CUDA graph holds every fit's whole damped GN step
 * (gn_step_graph's device-resident step, each fit an independent branch), so a
 * batched step is a single cudaGraphLaunch.  gn_batch_capture_graph captures it
 * for the parameter buffers thetas (host array of n_fits device pointers, in
 * place like gn_step; the addresses are part of the graph, so capture again
 * after changing any of them or any fit's precision or lambda setting) and
 * allocates the per-fit device states, capture streams and each fit's
 * workspace; it synchronises the device and must not be called while the
 * batch's fits have work in flight.  gn_batch_graph_step then runs one step of
 * every fit from the host values lambdas, dampings (in/out, as gn_batch_step);
 * a fit whose factorisation fails is retried with damping x10 by replaying its
 * own solve graph (at most 5 times).  infos, status as gn_batch_step (ms_phase
 * is not filled).  Returns GN_ERR_INVALID when no graph was captured.  Cites:
 * the paper's sweeps over lambda seeds and architectures (Methods,
 * "Identifying Admissible lambda Values"). */
int gn_batch_capture_graph(gn_batch* b, double* const* thetas);
int gn_batch_graph_step(gn_batch* b, double* lambdas, double* dampings, gn_step_info* infos, int* status);

/* One step of the paper's own optimiser (Methods, "Second-order Optimizer"): G is
 * estimated by an exponential moving average over iterations of the unbiased rank-1
 * estimate u u^T, u = J~^T v (v independent +-1 signs, E[v v^T] = I), and the step
 * d = alpha Delta + mu v_prev uses the learning rate and momentum that minimise the
 * quadratic model g.d + 1/2 d.(G + gamma I).d with the exact G applied through J~
 * products (Martens & Grosse 2015), Delta = -(G_ema + gamma I)^{-1} g.
 * G_ema: device [P' x P'] row-major, in/out (input ignored when first != 0: the average
 * starts at the first sample); v_prev: device [P'], the previous update d, in/out
 * (treated as 0 when first != 0); signs: device [rows] of +-1 values (caller-drawn);
 * beta: weight of the old average, in [0, 1).  theta, lambda, damping as gn_step; the
 * update is applied whenever the new loss is finite, and damping follows the same
 * Levenberg-Marquardt rule as gn_step (rho against the undamped model).  Needs the whole
 * Jacobian in the handle's J~ buffer (rows x P' x 8 bytes <= 32 GiB), else
 * GN_ERR_UNSUPPORTED.  Returns GN_OK, GN_WARN_NO_DECREASE (non-finite new loss: theta,
 * lambda kept, v_prev zeroed, damping x10), GN_ERR_NOT_SPD, GN_ERR_NONFINITE, GN_ERR_INVALID
 * or GN_ERR_CUDA.  Synchronises. */
int gn_step_ema(gn_handle* h, double* theta, double* lambda, double* damping, double* G_ema, double* v_prev,
                const double* signs, double beta, int first, gn_step_info* info);

/* ---- the blow-up rate lambda (Methods, "Identifying Admissible lambda Values") ---- */

/* trainable = 1 (default): lambda is an unknown of every step (column P of J~, entry P of
 * the gradients).  trainable = 0: lambda is held fixed, as funnel inference trains the
 * network at a constant lambda: column P of J~ and entry P of every gradient are zero, so
 * gn_step, gn_step_graph and gn_step_ema leave lambda unchanged (delta_P = 0 exactly).
 * Captured graphs are recaptured on the next gn_step_graph call; a batch graph keeps the
 * setting it was captured with.  GN_ERR_INVALID for other values. */
int gn_set_lambda_trainable(gn_handle* h, int trainable);

/* The lambda-inference rule (item 2): the self-similar equation differentiated at the
 * origin gives lambda from the current fields.  Boussinesq lambda = -3 - 2 d1 U1(0, 0)
 * (the rule the paper prints), IPM lambda = -2 - 2 d1 U1(0, 0) (U1 = d2 Psi, so d1 U1 =
 * d12 Psi), CCF lambda = -2 - 2 U'(0) with U'(0) = H[Theta/x](0) by the library's discrete
 * Hilbert operator; the IPM and CCF rules follow from the same steps on this library's
 * residual operators.  theta: device [P]; lambda: the value the network is evaluated at
 * (it enters q and the envelopes); *lambda_out: host.  Synchronises.  Returns
 * GN_ERR_UNSUPPORTED for Burgers (U'(0) = -1 for every lambda: the rule is empty),
 * GN_ERR_NONFINITE for a non-finite result. */
int gn_lambda_inference(gn_handle* h, const double* theta, double lambda, double* lambda_out);

/* The funnel-inference signal r_hat(lambda) (item 3): over the interior points with
 * |y| <= radius and all equations, the residual R_k (unweighted) of largest magnitude,
 * with its sign; ties go to the first point, then the first equation.  *r_hat (host) = 0
 * and *point = -1 when no point lies within radius; point (host, may be NULL) receives the
 * point index.  Overwrites the handle's residual buffer.  Synchronises. */
int gn_signed_max_residual(gn_handle* h, const double* theta, double lambda, double radius, double* r_hat,
                           int64_t* point);

/* The profile itself: the handle's network fields Phi_A (Eq. ansatz_vorticity and its
 * generalisation, envelopes included) at caller points.  y: device SoA [d][n]; out: device
 * [n][ld] with ld from gn_field_jets_ld: per field its value, gradient (d entries) and
 * Hessian (2D: d11, d12, d22; 1D: one 0), then for CCF the value of g = Theta / y.  In a
 * stage-2 handle these are Phi_2's fields (the composed profile is Phi_1 + eps Phi_2).
 * Asynchronous on the handle's stream.  Cites: Methods, "Solution Modeling". */
int gn_field_jets(gn_handle* h, const double* theta, double lambda, const double* y, int64_t n, double* out);
int gn_field_jets_ld(const gn_handle* h, int64_t* ld);

/* The funnel-inference update (item 3): n = 1: lambda_0 + dlambda; n >= 2: the secant zero
 * through the last two pairs, lambda_n - r_n (lambda_n - lambda_{n-1}) / (r_n - r_{n-1}).
 * The paper's printed update puts lambda_n in front of the correction anchored at
 * lambda_{n-1}; its text calls the update the secant formula, which is what this computes.
 * lambdas, r_hats: host [n]; *lambda_next: host.  Host arithmetic only (no GPU work).
 * GN_ERR_INVALID when n < 1 or r_n == r_{n-1}. */
int gn_funnel_next(const double* lambdas, const double* r_hats, int n, double dlambda, double* lambda_next);

/* Multi-stage training (Methods, "Multi-stage Training"): turn the handle into the
 * second stage of a fit whose first stage is the network (n_layers1, widths1, theta1) at
 * the fixed blow-up rate lambda.  From then on every field is Phi_1 + eps Phi_2, Phi_1
 * the frozen stage-1 network and Phi_2 the handle's own network (its own widths and
 * parameters), every row of r~ and J~ is divided by eps (the normalised stage-2 equation
 * R(Phi_1 + eps Phi_2) / eps = R_1 / eps + D[Phi_1] Phi_2 + O(eps), the paper's linearised
 * equation with its O(eps^2) part kept), lambda is held fixed (gn_set_lambda_trainable(0))
 * and gn_max_residual reports max |R_k| of the composed field.  Pass the same lambda to
 * every later call.  widths1: host [n_layers1 + 1] with widths1[0] = d and
 * widths1[n_layers1] = the number of fields; theta1: device [P1], read during the call only
 * (the stage-1 field jets at every point are evaluated once and kept, so later calls do not
 * read it); eps > 0, typically the stage-1 maximum residual.  Calling it again replaces
 * the first stage.  Synchronises.  GN_ERR_INVALID, GN_ERR_OOM or GN_ERR_CUDA. */
int gn_set_stage1(gn_handle* h, int n_layers1, const int* widths1, const double* theta1, double lambda, double eps);

/* Checkpoint and resume of a fit (the paper's fits run for many Gauss-Newton
 * steps; resuming one needs theta, lambda and the damping).  The file holds,
 * little-endian: the magic bytes "GNCK", a uint32 version (1), the int32
 * equation and n_layers, int32 widths[GN_MAX_LAYERS + 1], the int64 parameter
 * count P, the float64 lambda and damping, then theta as P float64 values.
 * gn_save: theta is device memory [P] (read), lambda and damping host values;
 * synchronises the handle's stream.  gn_load: checks the file against the
 * handle's equation and widths (GN_ERR_MISMATCH otherwise), writes theta
 * (device [P]) and *lambda, *damping (host).  Both return GN_OK, GN_ERR_INVALID,
 * GN_ERR_IO, GN_ERR_MISMATCH (load) or GN_ERR_CUDA; the caller owns all buffers. */
int gn_save(gn_handle* h, const char* path, const double* theta, double lambda, double damping);
int gn_load(gn_handle* h, const char* path, double* theta, double* lambda, double* damping);

/* Max |R_k| over the interior points (Methods, "Validation Metrics", max d0
 * residual) at (theta, lambda), unweighted.  *out: host.  Synchronises. */
int gn_max_residual(gn_handle* h, const double* theta, double lambda, double* out);

/* g_out[0..ncols) = J^T r without a handle and without allocating anything.
 * The paper has no counterpart: this is a service for callers that cannot
 * call cudaMalloc (a host application that owns all device memory through its
 * own allocator, loops that must avoid the synchronisation an allocation may
 * imply, plug-ins that only receive device pointers).  J: device, row-major
 * [nrows x ld] with ncols <= ld used columns; r: device [nrows]; g_out:
 * device [ncols]; all caller-owned.  Work is queued on cuda_stream (a
 * cudaStream_t, NULL = legacy default stream); the call does not synchronise.
 * Scratch lives in a fixed 8 MiB device array inside the library image,
 * held by every GPU that loads the library until the process exits;
 * ncols > 16384 returns GN_ERR_TOO_LARGE.  The first call on a device looks
 * up the array's device address (make it before any stream capture); that
 * address stays cached and is not valid after a cudaDeviceReset of the device,
 * so do not call this entry point on a device after resetting it.  All
 * calls on a device share the array: calls that overlap on the GPU race, so
 * serialise them.  Returns GN_OK, GN_ERR_INVALID, GN_ERR_TOO_LARGE,
 * GN_ERR_UNSUPPORTED (device index >= 64) or GN_ERR_CUDA. */
int gn_jtr_noalloc(const double* J, int64_t ld, int64_t nrows, int64_t ncols, const double* r, double* g_out,
                   void* cuda_stream);

/* Testing hook of the failure path GN_ERR_TIMEOUT (no paper counterpart).  Every wait of the
 * split-precision tensor-core kernels on an mbarrier (a copy landing, an MMA completing, an
 * accumulator becoming free) is bounded in time; when one runs out, the kernel raises a
 * status bit, lets its copies and MMAs in flight finish (again with a bound), releases its
 * tensor memory and returns, and the calling entry point returns GN_ERR_TIMEOUT with the
 * CUDA context still usable.  wait_ns sets that bound for later launches (0 restores the
 * default of 4 s); starve_copies != 0 makes the kernels' producer issue no copies at all,
 * so no copy or MMA is ever in flight and every consumer's wait runs out after wait_ns,
 * which lets a test exercise the path without any fault.  Process-wide; not for use while
 * other threads launch work.  Returns GN_OK. */
int gn_test_bounded_waits(unsigned long long wait_ns, int starve_copies);

/* Number of CUDA kernels this library has launched in this process so far
 * (a diagnostic counter; read it before and after a region to count its launches). */
int64_t gn_kernel_launches(void);

/* Where the last GN_ERR_CUDA / GN_ERR_UNSUPPORTED of this host thread came
 * from ("file:line: CUDA message"); empty if none.  Static storage, per thread. */
const char* gn_last_error_detail(void);

/* Static message for a status code. */
const char* gn_error_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* GN_H_ */
