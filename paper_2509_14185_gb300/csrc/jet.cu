// Fused per-point kernel: Taylor jets through the tanh MLP -> self-similar
// residual -> weighted Jacobian row (or residual only, or adjoint gradient).
//
// Paper references (Methods): the ansatz phi_A = (1-t)^{k_A} Phi_A(y),
// y = x/(1-t)^{1+lambda} (Eq. self-similar); the compactified inputs
// q = (1+|y|^2)^{-1/(2(1+lambda))}, beta = y2/sqrt(1+|y|^2) and the
// symmetry x network x decay envelope (Eq. ansatz_vorticity, generalised to
// every field); the tanh MLP ("Solution Modeling"); the residuals R_k of the
// static equations (Eq. self-similar-static) and the d0 loss with weights rho
// ("Training Loss"); the Jacobian rows feed the Gauss-Newton matrix
// ("Second-order Optimizer").  lambda is an unknown: column P of J~ is the
// total derivative dR/dlambda (through q, the envelope exponents and the
// explicit lambda terms).
//
// Work decomposition (one warp per point, grid-stride over points):
//  1. forward: jets of the network output in the network inputs z = q (1D:
//     value, d/dq, d2/dq2) or z = (q, beta) (2D: value, first, second and the
//     third derivatives along q that the lambda column needs).  Lanes own
//     output neurons; the transposed weights are read coalesced from global
//     memory (they stay in L1/L2), activations live in per-warp shared memory.
//  2. residual: every lane evaluates the residual chain in dual numbers; lane
//     0 carries the tangent along lambda, lane 1 + f*C_R + c the tangent along
//     network output f, jet component c.  One pass therefore yields R_k,
//     dR_k/dlambda and the reverse-pass seeds dR_k/d(output jets).
//  3. reverse: per row, the seeds are pulled back through the jet
//     nonlinearity and the layers; weight-gradient entries
//     sum_c abar_c[o] h_c[i] are written as consecutive addresses by
//     consecutive lanes (coalesced J row stores), or accumulated into a
//     per-warp partial gradient (adjoint mode).
#include <cmath>

#include "gn_internal.cuh"

namespace gn {
namespace {

// Grid cap: two resident blocks per SM keep the FP64 pipe busy (the kernel is
// FP64-bound); it also bounds the per-warp partial-gradient buffer.
constexpr int64_t kJetMaxBlocks = 152 * 2;

struct Dl {
  double v, d;
};
__device__ __forceinline__ Dl operator+(Dl a, Dl b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dl operator-(Dl a, Dl b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dl operator-(Dl a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dl operator*(Dl a, Dl b) { return {a.v * b.v, fma(a.v, b.d, a.d * b.v)}; }
__device__ __forceinline__ Dl operator*(double s, Dl a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dl operator+(double s, Dl a) { return {s + a.v, a.d}; }
__device__ __forceinline__ Dl dconst(double v) { return {v, 0.0}; }
// u^e for a constant base u > 0 and a dual exponent e.
__device__ __forceinline__ Dl pow_cb(double u, Dl e) {
  const double lu = log(u);
  const double p = exp(e.v * lu);
  return {p, p * lu * e.d};
}

template <int EQ> struct Eq;
template <> struct Eq<GN_BURGERS> { static constexpr int D = 1, NF = 1, NE = 1; };
template <> struct Eq<GN_CCF> { static constexpr int D = 1, NF = 1, NE = 1; };
template <> struct Eq<GN_IPM> { static constexpr int D = 2, NF = 2, NE = 2; };
template <> struct Eq<GN_BOUSSINESQ> { static constexpr int D = 2, NF = 3, NE = 3; };

// Network-input jet components.  1D: (v, z, zz).  2D: (v, q, b, qq, qb, bb,
// qqq, qqb, qbb).  The reverse pass uses the first C_R of them.
template <int D> struct JT;
template <> struct JT<1> { static constexpr int CR = 2, CF = 3; };
template <> struct JT<2> { static constexpr int CR = 6, CF = 9; };

// Component reached by one more derivative along q (used for d/dlambda,
// since lambda enters the network only through q).
template <int D> __device__ __forceinline__ int q_shift(int c);
template <> __device__ __forceinline__ int q_shift<1>(int c) { return c + 1; }
template <> __device__ __forceinline__ int q_shift<2>(int c) {
  // v->q, q->qq, b->qb, qq->qqq, qb->qqb, bb->qbb
  const int m[6] = {1, 3, 4, 6, 7, 8};
  return m[c];
}

// y-jet of dual numbers: value, first derivatives, second derivatives
// (1D: h[0] = d11; 2D: h[0] = d11, h[1] = d12, h[2] = d22).
template <int D> struct YJ {
  Dl v;
  Dl g[D];
  Dl h[D == 1 ? 1 : 3];
};
template <int D> __device__ __forceinline__ int hix(int i, int j) { return D == 1 ? 0 : i + j; }

template <int D> __device__ __forceinline__ YJ<D> ymul(const YJ<D>& a, const YJ<D>& b) {
  YJ<D> c;
  c.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < D; i++) c.g[i] = a.g[i] * b.v + a.v * b.g[i];
#pragma unroll
  for (int i = 0; i < D; i++)
#pragma unroll
    for (int j = i; j < D; j++) {
      const int k = hix<D>(i, j);
      c.h[k] = a.h[k] * b.v + a.g[i] * b.g[j] + a.g[j] * b.g[i] + a.v * b.h[k];
    }
  return c;
}

// Envelope y1^m * u^e (u = 1 + |y|^2) as a y-jet; e is a dual number.
//   (u^e)_i = 2 e y_i u^e / u,  (u^e)_ij = 2 e u^e / u (delta_ij + 2 (e-1) y_i y_j / u).
template <int D> __device__ YJ<D> envelope(const double* y, double u, int m, Dl e) {
  const Dl W = pow_cb(u, e);
  const double iu = 1.0 / u;
  const Dl c1 = (2.0 * iu) * (e * W);  // 2 e W / u
  YJ<D> Wj;
  Wj.v = W;
#pragma unroll
  for (int i = 0; i < D; i++) Wj.g[i] = y[i] * c1;
  const Dl em1 = e + dconst(-1.0);
#pragma unroll
  for (int i = 0; i < D; i++)
#pragma unroll
    for (int j = i; j < D; j++) {
      const Dl inner = dconst(i == j ? 1.0 : 0.0) + (2.0 * y[i] * y[j] * iu) * em1;
      Wj.h[hix<D>(i, j)] = c1 * inner;
    }
  if (m == 0) return Wj;
  YJ<D> Y;
  const double y1 = y[0];
  Y.v = dconst(m == 1 ? y1 : y1 * y1);
#pragma unroll
  for (int i = 0; i < D; i++) Y.g[i] = dconst(0.0);
  Y.g[0] = dconst(m == 1 ? 1.0 : 2.0 * y1);
#pragma unroll
  for (int k = 0; k < (D == 1 ? 1 : 3); k++) Y.h[k] = dconst(0.0);
  Y.h[0] = dconst(m == 1 ? 0.0 : 2.0);
  return ymul<D>(Y, Wj);
}

// Exponential output map on one field's jet components a[0 .. CF) (value, q, (b,) the second
// orders, the q-direction third orders the lambda column needs): N = exp(a) by the chain rule,
// every component exp(a_v) times the complete Bell polynomial of the a-derivatives.
template <int D, int CF>
__device__ __forceinline__ void exp_jet(const double* a, double* N) {
  const double E = exp(a[0]);
  N[0] = E;
  if constexpr (D == 1) {
    N[1] = E * a[1];
    if constexpr (CF > 2) N[2] = E * (a[2] + a[1] * a[1]);
  } else {
    const double q = a[1], b = a[2];
    N[1] = E * q;
    N[2] = E * b;
    N[3] = E * (a[3] + q * q);
    N[4] = E * (a[4] + q * b);
    N[5] = E * (a[5] + b * b);
    if constexpr (CF > 6) {
      N[6] = E * (a[6] + 3.0 * q * a[3] + q * q * q);
      N[7] = E * (a[7] + b * a[3] + 2.0 * q * a[4] + q * q * b);
      N[8] = E * (a[8] + q * a[5] + 2.0 * b * a[4] + q * b * b);
    }
  }
}

// Its adjoint on the components the reverse pass carries (c < C_R): nb holds dN-bar on entry
// and the pre-activation adjoints a-bar_c = sum_k N-bar_k dN_k / da_c on exit.
template <int D>
__device__ __forceinline__ void exp_jet_adjoint(const double* a, double* nb) {
  const double E = exp(a[0]);
  if constexpr (D == 1) {
    const double a0 = nb[0] * E + nb[1] * (E * a[1]);
    nb[1] = nb[1] * E;
    nb[0] = a0;
  } else {
    const double q = a[1], b = a[2];
    const double N[6] = {E, E * q, E * b, E * (a[3] + q * q), E * (a[4] + q * b), E * (a[5] + b * b)};
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 6; c++) s = fma(nb[c], N[c], s);
    const double a1 = E * (nb[1] + 2.0 * q * nb[3] + b * nb[4]);
    const double a2 = E * (nb[2] + q * nb[4] + 2.0 * b * nb[5]);
    nb[0] = s;
    nb[1] = a1;
    nb[2] = a2;
    nb[3] *= E;
    nb[4] *= E;
    nb[5] *= E;
  }
}

// Per-warp shared-memory layout (doubles).  H[j][c][ldw] for c < C_R: j = 0 network
// input, j = 1..L-1 outputs of hidden layers (the reverse pass reads them); the forward-only
// components c >= C_R (the third order the lambda column needs) of layer j live in a
// two-layer ping-pong X[j & 1][c - C_R][ldw]; AS[l][c-1][ldw] derivative components of
// hidden pre-activations; BA, BB [C_R][ldw] adjoint ping-pong; NN [NF][CF]; with the exponential
// output map NA [NF][CF], the last layer's own jets.
__host__ __device__ inline int64_t jet_smem_doubles(const NetDesc& net, int CF, int CR, int NF) {
  const int64_t ldw = net.maxw;
  return (int64_t)net.L * CR * ldw + 2 * (int64_t)(CF - CR) * ldw + (int64_t)(net.L - 1) * (CR - 1) * ldw +
         2 * (int64_t)CR * ldw + (int64_t)NF * CF + (net.exp_out ? (int64_t)NF * CF : 0) + 2;
}

// XO: the exponential output map (a separate instantiation, so the linear map's kernels carry
// none of its registers).  Occupancy is set by the per-warp shared memory: two blocks of eight
// warps per SM in 1D, one block in 2D, which the register budget states (<= 128 / 255).
template <int EQ, int MODE, bool XO>
__global__ void __launch_bounds__(256, Eq<EQ>::D == 1 ? 2 : 1) jet_kernel(const JetArgs A) {
  constexpr int D = Eq<EQ>::D, NF = Eq<EQ>::NF, NE = Eq<EQ>::NE;
  constexpr int CR = JT<D>::CR;
  constexpr int CF = (MODE == MODE_RESIDUAL) ? CR : JT<D>::CF;
  const NetDesc& net = A.net;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int ldw = net.maxw;
  const int L = net.L;
  extern __shared__ double sm[];
  double* base = sm + (int64_t)warp * jet_smem_doubles(net, CF, CR, NF);
  double* H = base;
  double* XH = H + (int64_t)L * CR * ldw;               // forward-only components, ping-pong
  double* AS = XH + 2 * (int64_t)(CF - CR) * ldw;
  // component c of layer j's jets
  auto hc = [&](int j, int c) -> double* {
    return c < CR ? H + ((int64_t)j * CR + c) * ldw : XH + ((int64_t)(j & 1) * (CF - CR) + (c - CR)) * ldw;
  };
  double* BA = AS + (int64_t)(L - 1) * (CR - 1) * ldw;
  double* BB = BA + CR * ldw;
  double* NN = BB + CR * ldw;
  double* NA = NN + NF * CF;   // the last layer's own jets under the exponential output map

  const int kind = A.kind;
  const int nrow = (kind == KIND_INTERIOR) ? NE : 1;
  const int64_t gw = (int64_t)blockIdx.x * wpb + warp;
  const int64_t nw = (int64_t)gridDim.x * wpb;
  double* gp = (MODE == MODE_GRADIENT) ? A.gpart + gw * A.ldg : nullptr;
  const double lam = A.lamp ? *A.lamp : A.lam;
  const int K = 1 + NF * CR;                  // tangent directions in use
  const int dir = (lane < K) ? lane : 0;      // this lane's direction

  for (int64_t pt = gw; pt < A.n; pt += nw) {
    double y[D];
#pragma unroll
    for (int k = 0; k < D; k++) y[k] = A.y[(int64_t)k * A.ystride + pt];
    double u = 1.0;
#pragma unroll
    for (int k = 0; k < D; k++) u = fma(y[k], y[k], u);
    // a = 1/(1+lambda), q = u^{-a/2}
    const Dl a = {1.0 / (1.0 + lam), (dir == 0 && MODE != MODE_RESIDUAL) ? -1.0 / ((1.0 + lam) * (1.0 + lam)) : 0.0};
    const Dl q = pow_cb(u, -0.5 * a);
    double beta = 0.0;
    if (D == 2) beta = y[1] / sqrt(u);

    // ---- 1. network input jets ------------------------------------------
    for (int idx = lane; idx < CR * ldw; idx += 32) H[idx] = 0.0;
    for (int idx = lane; idx < (CF - CR) * ldw; idx += 32) XH[idx] = 0.0;
    __syncwarp();
    if (lane == 0) {
      H[0 * ldw + 0] = q.v;
      H[1 * ldw + 0] = 1.0;           // d q / d q
      if (D == 2) {
        H[0 * ldw + 1] = beta;
        H[2 * ldw + 1] = 1.0;         // d beta / d beta
      }
    }
    __syncwarp();

    // ---- 2. forward through the layers ------------------------------------
    for (int l = 0; l < L; l++) {
      const int in = net.w[l], out = net.w[l + 1];
      const double* hinc[CF];
#pragma unroll
      for (int c = 0; c < CF; c++) hinc[c] = hc(l, c);
      const double* wtl = A.wt + net.offT[l];
      const bool fixed = net.fourier && l == 1;   // the Fourier map: no bias, not in theta
      const double* bl = A.theta + net.offB[l];
      for (int o = lane; o < out; o += 32) {
        double acc[CF];
        acc[0] = fixed ? 0.0 : bl[o];
#pragma unroll
        for (int c = 1; c < CF; c++) acc[c] = 0.0;
        for (int i = 0; i < in; i++) {
          const double wv = __ldg(wtl + (int64_t)i * out + o);
#pragma unroll
          for (int c = 0; c < CF; c++) acc[c] = fma(wv, hinc[c][i], acc[c]);
        }
        if (l < L - 1) {
          double* hoc[CF];
#pragma unroll
          for (int c = 0; c < CF; c++) hoc[c] = hc(l + 1, c);
          double* ao = AS + (int64_t)l * (CR - 1) * ldw;
          // activation and its first three derivatives: tanh; identity on a Fourier
          // network's linear input layer; cos / sin on its Fourier layer's two halves
          double t, t1, t2, t3;
          if (net.fourier && l == 0) {
            t = acc[0]; t1 = 1.0; t2 = 0.0; t3 = 0.0;
          } else if (fixed) {
            double sn, cs;
            sincos(acc[0], &sn, &cs);
            if (o < out / 2) { t = cs; t1 = -sn; t2 = -cs; t3 = sn; }
            else { t = sn; t1 = cs; t2 = -sn; t3 = -cs; }
          } else {
            t = tanh(acc[0]);
            t1 = 1.0 - t * t;
            t2 = -2.0 * t * t1;
            t3 = -2.0 * t1 * t1 - 2.0 * t * t2;
          }
          hoc[0][o] = t;
          if (D == 1) {
            hoc[1][o] = t1 * acc[1];
            if (CF > 2) hoc[2][o] = t2 * acc[1] * acc[1] + t1 * acc[2];
            ao[o] = acc[1];
          } else {
            const double aq = acc[1], ab = acc[2], aqq = acc[3], aqb = acc[4], abb = acc[5];
            hoc[1][o] = t1 * aq;
            hoc[2][o] = t1 * ab;
            hoc[3][o] = t2 * aq * aq + t1 * aqq;
            hoc[4][o] = t2 * aq * ab + t1 * aqb;
            hoc[5][o] = t2 * ab * ab + t1 * abb;
            if (CF > 6) {
              hoc[6][o] = t3 * aq * aq * aq + 3.0 * t2 * aq * aqq + t1 * acc[6];
              hoc[7][o] = t3 * aq * aq * ab + t2 * (2.0 * aq * aqb + ab * aqq) + t1 * acc[7];
              hoc[8][o] = t3 * aq * ab * ab + t2 * (2.0 * ab * aqb + aq * abb) + t1 * acc[8];
            }
#pragma unroll
            for (int c = 1; c < 6; c++) ao[(c - 1) * ldw + o] = acc[c];
          }
        } else {
#pragma unroll
          for (int c = 0; c < CF; c++) NN[o * CF + c] = acc[c];
        }
      }
      __syncwarp();
    }

    // exponential output map: NN becomes exp of the last layer's jets, which NA keeps for the
    // reverse pass
    if constexpr (XO) {
      if (lane < NF) {
#pragma unroll
        for (int c = 0; c < CF; c++) NA[lane * CF + c] = NN[lane * CF + c];
        exp_jet<D, CF>(NA + lane * CF, NN + lane * CF);
      }
      __syncwarp();
    }

    // ---- 3. residual chain in dual numbers ---------------------------------
    // network output jets as duals along this lane's direction
    Dl nn[NF][CR];
#pragma unroll
    for (int f = 0; f < NF; f++)
#pragma unroll
      for (int c = 0; c < CR; c++) {
        double dv = 0.0;
        if (MODE != MODE_RESIDUAL) {
          if (dir == 0) dv = NN[f * CF + q_shift<D>(c)] * q.d;
          else if (dir == 1 + f * CR + c) dv = 1.0;
        }
        nn[f][c] = {NN[f * CF + c], dv};
      }
    // q jets: q_i = -a y_i q / u ; q_ij = -a q / u (delta_ij - (a+2) y_i y_j / u)
    const double iu = 1.0 / u;
    Dl qg[D], qh[D == 1 ? 1 : 3];
    const Dl aq_u = (-iu) * (a * q);
#pragma unroll
    for (int i = 0; i < D; i++) qg[i] = y[i] * aq_u;
#pragma unroll
    for (int i = 0; i < D; i++)
#pragma unroll
      for (int j = i; j < D; j++)
        qh[hix<D>(i, j)] = aq_u * (dconst(i == j ? 1.0 : 0.0) + (-y[i] * y[j] * iu) * (a + dconst(2.0)));
    // beta jets (2D): beta_1 = -y1 y2 u^-3/2, beta_2 = (1+y1^2) u^-3/2,
    // beta_11 = y2 (3 y1^2 - u) u^-5/2, beta_12 = y1 (3 y2^2 - u) u^-5/2,
    // beta_22 = -3 y2 (1 + y1^2) u^-5/2
    double bg[2] = {0.0, 0.0}, bh[3] = {0.0, 0.0, 0.0};
    if (D == 2) {
      const double s3 = iu / sqrt(u), s5 = s3 * iu;
      bg[0] = -y[0] * y[1] * s3;
      bg[1] = (1.0 + y[0] * y[0]) * s3;
      bh[0] = y[1] * (3.0 * y[0] * y[0] - u) * s5;
      bh[1] = y[0] * (3.0 * y[1] * y[1] - u) * s5;
      bh[2] = -3.0 * y[1] * (1.0 + y[0] * y[0]) * s5;
    }
    const Dl lamd = {lam, (dir == 0 && MODE != MODE_RESIDUAL) ? 1.0 : 0.0};
    // fields F_f = E_f * N_f
    YJ<D> F[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) {
      YJ<D> N;
      N.v = nn[f][0];
      if (D == 1) {
        N.g[0] = nn[f][1] * qg[0];
        N.h[0] = dconst(0.0);  // not used by the 1D residuals
      } else {
#pragma unroll
        for (int i = 0; i < D; i++) N.g[i] = nn[f][1] * qg[i] + bg[i] * nn[f][2];
#pragma unroll
        for (int i = 0; i < D; i++)
#pragma unroll
          for (int j = i; j < D; j++) {
            const int k = hix<D>(i, j);
            N.h[k] = nn[f][3] * (qg[i] * qg[j]) + nn[f][4] * (bg[j] * qg[i] + bg[i] * qg[j]) +
                     (bg[i] * bg[j]) * nn[f][5] + nn[f][1] * qh[k] + bh[k] * nn[f][2];
          }
      }
      // exponent k_f(lambda) and prefactor (y1^m, extra power of u)
      Dl kf;
      int m;
      double e0;
      if (EQ == GN_BURGERS) { kf = lamd; m = 1; e0 = -0.5; }
      else if (EQ == GN_CCF) { kf = lamd; m = 2; e0 = -1.0; }
      else if (EQ == GN_IPM) {
        if (f == 0) { kf = lamd; m = 0; e0 = 0.0; }
        else { kf = dconst(1.0) + 2.0 * lamd; m = 1; e0 = -0.5; }
      } else {
        if (f == 0) { kf = dconst(-1.0); m = 1; e0 = -0.5; }
        else if (f == 1) { kf = lamd + dconst(-1.0); m = 0; e0 = 0.0; }
        else { kf = dconst(1.0) + 2.0 * lamd; m = 1; e0 = -0.5; }
      }
      const Dl e = dconst(e0) + 0.5 * (kf * a);
      F[f] = ymul<D>(envelope<D>(y, u, m, e), N);
    }
    constexpr int NJ = 1 + D + (D == 1 ? 1 : 3);   // probe values per field

    if (kind == KIND_PROBE) {
      // field jets at the point: value, gradient and (2D) Hessian (d11, d12, d22) per field;
      // the 1D kernels carry no second y-derivative of the fields, so 1D writes 0 there;
      // CCF adds g = Theta / y (the Hilbert operator's integrand)
      if (lane == 0 && A.r) {
        double* o = A.r + pt * (NF * NJ + (EQ == GN_CCF ? 1 : 0));
#pragma unroll
        for (int f = 0; f < NF; f++) {
          o[f * NJ] = F[f].v.v;
#pragma unroll
          for (int i = 0; i < D; i++) o[f * NJ + 1 + i] = F[f].g[i].v;
#pragma unroll
          for (int k = 0; k < (D == 1 ? 1 : 3); k++) o[f * NJ + 1 + D + k] = (D == 1) ? 0.0 : F[f].h[k].v;
        }
        if (EQ == GN_CCF) {
          const YJ<D> Eg = envelope<D>(y, u, 1, dconst(-1.0) + 0.5 * (lamd * a));
          o[NF * NJ] = (Eg.v * nn[0][0]).v;
        }
      }
      continue;
    }

    // stage 2: Phi = Phi_1 + eps Phi_2, Phi_1 a constant (its jets precomputed at this point)
    if (A.base && kind != KIND_NODE) {
      const double* b = A.base + pt * A.base_ld;
      const double ep = A.eps;
#pragma unroll
      for (int f = 0; f < NF; f++) {
        F[f].v = Dl{b[f * NJ] + ep * F[f].v.v, ep * F[f].v.d};
#pragma unroll
        for (int i = 0; i < D; i++) F[f].g[i] = Dl{b[f * NJ + 1 + i] + ep * F[f].g[i].v, ep * F[f].g[i].d};
#pragma unroll
        for (int k = 0; k < (D == 1 ? 1 : 3); k++)
          F[f].h[k] = Dl{b[f * NJ + 1 + D + k] + ep * F[f].h[k].v, ep * F[f].h[k].d};
      }
    }

    // residuals (or the single value of a wall/node/norm row)
    Dl R[NE];
    double sUv = 0.0;
    const Dl opl = dconst(1.0) + lamd;
    if (kind == KIND_INTERIOR) {
      if (EQ == GN_BURGERS) {
        const YJ<D>& U = F[0];
        R[0] = (-1.0) * (lamd * U.v) + (y[0] * opl + U.v) * U.g[0];
      } else if (EQ == GN_CCF) {
        // U = sum_j K_ij g_j + D_i g(y_i); the K part's d/dlambda is added by
        // the Hilbert contraction (it carries the lambda column of J_g).
        const YJ<D> Eg = envelope<D>(y, u, 1, dconst(-1.0) + 0.5 * (lamd * a));
        Dl gi = Eg.v * nn[0][0];
        if (A.base) gi = Dl{A.base[pt * A.base_ld + NF * NJ] + A.eps * gi.v, A.eps * gi.d};
        const Dl Uv = dconst(A.ug[pt]) + A.dcoef[pt] * gi;
        const YJ<D>& T = F[0];
        R[0] = (-1.0) * (lamd * T.v) + (y[0] * opl + Uv) * T.g[0];
        sUv = T.g[0].v;
      } else if (EQ == GN_IPM) {
        const YJ<D>& P = F[0];
        const YJ<D>& S = F[1];
        const Dl V1 = y[0] * opl + S.g[1];
        const Dl V2 = y[D - 1] * opl + (-S.g[0]);
        R[0] = (-1.0) * (lamd * P.v) + V1 * P.g[0] + V2 * P.g[D - 1];
        R[NE > 1 ? 1 : 0] = S.h[0] + S.h[D == 1 ? 0 : 2] - P.g[0];
      } else {
        const YJ<D>& Om = F[0];
        const YJ<D>& Th = F[NF > 1 ? 1 : 0];
        const YJ<D>& S = F[NF - 1];
        const Dl V1 = y[0] * opl + S.g[D - 1];
        const Dl V2 = y[D - 1] * opl + (-S.g[0]);
        R[0] = Om.v + V1 * Om.g[0] + V2 * Om.g[D - 1] - Th.g[0];
        R[NE > 1 ? 1 : 0] = (dconst(1.0) - lamd) * Th.v + V1 * Th.g[0] + V2 * Th.g[D - 1];
        R[NE > 2 ? 2 : 0] = S.h[0] + S.h[D == 1 ? 0 : 2] + Om.v;
      }
    } else if (kind == KIND_WALL) {
      R[0] = F[NF - 1].v;
    } else if (kind == KIND_NORM || kind == KIND_INF || kind == KIND_RELU) {
      // normalisation: Phi_A0 or its d/dy1 minus the target; decay: Phi_A0 itself; bound:
      // relu(s (Phi_A0 - b)), zero (with a zero derivative) while the bound holds
      Dl val = F[0].v, dy1 = F[0].g[0];
#pragma unroll
      for (int f = 1; f < NF; f++)   // constant register indices only
        if (f == A.nfield) {
          val = F[f].v;
          dy1 = F[f].g[0];
        }
      R[0] = (kind == KIND_NORM && A.nderiv) ? dy1 : val;
      R[0].v -= A.c_norm;
      if (kind == KIND_RELU) {
        R[0] = (double)A.rsign * R[0];
        if (!(R[0].v > 0.0)) R[0] = Dl{0.0, 0.0};
      }
    } else {  // KIND_NODE (CCF): g = y/u * NN * q^{-lambda}
      const YJ<D> Eg = envelope<D>(y, u, 1, dconst(-1.0) + 0.5 * (lamd * a));
      R[0] = Eg.v * nn[0][0];
      if (A.base) R[0] = Dl{A.base[pt] + A.eps * R[0].v, A.eps * R[0].d};
    }

    // ---- 4. rows ------------------------------------------------------------
    double w = A.wscale;
    if (kind == KIND_INTERIOR && A.rho) w *= sqrt(A.rho[pt]);
    const int64_t rbase = A.row0 + pt * nrow;
    for (int e = 0; e < nrow; e++) {
      const double rv = w * R[e].v;
      if (lane == 0) {
        if (A.r) A.r[rbase + e] = rv;
        if (!isfinite(rv)) atomicOr(A.flag, 1);
      }
    }
    if (EQ == GN_CCF && kind == KIND_INTERIOR && A.sU && lane == 0 && MODE != MODE_GRADIENT) A.sU[pt] = w * sUv;
    if (MODE == MODE_RESIDUAL) continue;

    // seeds for the reverse pass: one per row (Jacobian) or combined (gradient)
    int nrev = (MODE == MODE_GRADIENT) ? 1 : nrow;
    double comb[NE];
#pragma unroll
    for (int e = 0; e < NE; e++) comb[e] = 0.0;
    if (MODE == MODE_GRADIENT) {
      for (int e = 0; e < nrow; e++) comb[e] = A.seed ? A.seed[rbase + e] : w * R[e].v;
      if (EQ == GN_CCF && kind == KIND_INTERIOR && A.sU && lane == 0) A.sU[pt] = comb[0] * w * sUv;
    }
    for (int e = 0; e < nrev; e++) {
      const int64_t row = rbase + e;
      double* Jrow = nullptr;
      if (MODE == MODE_JACOBIAN) {
        if (row < A.jrow_lo || row >= A.jrow_hi) continue;
        Jrow = A.J + (row - A.jrow_lo) * A.ldJ;
      }
      // seed of this lane's direction, and d/dlambda (lane 0)
      double sd;
      if (MODE == MODE_GRADIENT) {
        sd = 0.0;
        for (int ee = 0; ee < nrow; ee++) sd += comb[ee] * w * R[ee].d;
      } else {
        sd = w * R[e].d;
      }
      if (lane == 0) {   // the lambda column (zero while lambda is held fixed)
        if (MODE == MODE_JACOBIAN) Jrow[net.P] = A.lam_frozen ? 0.0 : sd;
        else if (!A.lam_frozen) gp[net.P] += sd;
      }
      if (lane >= 1 && lane < K) {
        const int f = (lane - 1) / CR, c = (lane - 1) % CR;
        BA[c * ldw + f] = sd;
      }
      __syncwarp();
      if constexpr (XO) {   // through the output map to the last layer's own jets
        if (lane < NF) {
          double nb[CR];
#pragma unroll
          for (int c = 0; c < CR; c++) nb[c] = BA[c * ldw + lane];
          exp_jet_adjoint<D>(NA + lane * CF, nb);
#pragma unroll
          for (int c = 0; c < CR; c++) BA[c * ldw + lane] = nb[c];
        }
        __syncwarp();
      }
      double* ab = BA;
      double* hb = BB;
      for (int l = L - 1; l >= 0; l--) {
        const int in = net.w[l], out = net.w[l + 1];
        const double* hin = H + (int64_t)l * CR * ldw;   // components c < C_R, ldw apart
        // weight and bias entries: W_l[o][i] = sum_c abar_c[o] h_c[i]; b_l[o] = abar_v[o]
        const int64_t nW = (int64_t)out * in;
        const int64_t off = net.offW[l];
        const bool fixed = net.fourier && l == 1;   // no parameters: no J columns
        for (int64_t idx = lane; idx < (fixed ? 0 : nW + out); idx += 32) {
          double v;
          if (idx < nW) {
            const int o = (int)(idx / in);
            const int i = (int)(idx - (int64_t)o * in);
            v = 0.0;
#pragma unroll
            for (int c = 0; c < CR; c++) v = fma(ab[c * ldw + o], hin[c * ldw + i], v);
          } else {
            v = ab[idx - nW];
          }
          if (MODE == MODE_JACOBIAN) Jrow[off + idx] = v;
          else gp[off + idx] += v;
        }
        if (l == 0) break;
        // hbar_c[i] = sum_o W_l[o][i] abar_c[o]
        const double* Wl = fixed ? A.fW : A.theta + off;
        for (int i = lane; i < in; i += 32) {
          double acc[CR];
#pragma unroll
          for (int c = 0; c < CR; c++) acc[c] = 0.0;
          for (int o = 0; o < out; o++) {
            const double wv = __ldg(Wl + (int64_t)o * in + i);
#pragma unroll
            for (int c = 0; c < CR; c++) acc[c] = fma(wv, ab[c * ldw + o], acc[c]);
          }
          // pull back through the activation jet of hidden layer l-1 (output H[l]): its
          // derivatives from the stored outputs (tanh: t; Fourier: the cos/sin pair)
          double t1, t2, t3;
          if (net.fourier && l - 1 == 0) {
            t1 = 1.0; t2 = 0.0; t3 = 0.0;
          } else if (net.fourier && l - 1 == 1) {
            const int half = in / 2;
            if (i < half) { const double cs = hin[i], sn = hin[i + half]; t1 = -sn; t2 = -cs; t3 = sn; }
            else { const double sn = hin[i], cs = hin[i - half]; t1 = cs; t2 = -sn; t3 = -cs; }
          } else {
            const double t = hin[i];
            t1 = 1.0 - t * t;
            t2 = -2.0 * t * t1;
            t3 = -2.0 * t1 * t1 - 2.0 * t * t2;
          }
          const double* as = AS + (int64_t)(l - 1) * (CR - 1) * ldw;
          if (D == 1) {
            const double az = as[i];
            hb[i] = acc[0] * t1 + acc[1] * t2 * az;
            hb[ldw + i] = acc[1] * t1;
          } else {
            const double aq = as[i], abv = as[ldw + i], aqq = as[2 * ldw + i], aqb = as[3 * ldw + i],
                         abb = as[4 * ldw + i];
            hb[i] = acc[0] * t1 + acc[1] * t2 * aq + acc[2] * t2 * abv + acc[3] * (t3 * aq * aq + t2 * aqq) +
                    acc[4] * (t3 * aq * abv + t2 * aqb) + acc[5] * (t3 * abv * abv + t2 * abb);
            hb[1 * ldw + i] = acc[1] * t1 + 2.0 * acc[3] * t2 * aq + acc[4] * t2 * abv;
            hb[2 * ldw + i] = acc[2] * t1 + acc[4] * t2 * aq + 2.0 * acc[5] * t2 * abv;
            hb[3 * ldw + i] = acc[3] * t1;
            hb[4 * ldw + i] = acc[4] * t1;
            hb[5 * ldw + i] = acc[5] * t1;
          }
        }
        __syncwarp();
        double* tmp = ab;
        ab = hb;
        hb = tmp;
      }
      __syncwarp();
    }
  }
}

__global__ void transpose_weights_kernel(const NetDesc net, const double* __restrict__ theta, double* wt) {
  for (int l = 0; l < net.L; l++) {
    if (net.fourier && l == 1) continue;   // the fixed Fourier layer's copy is written once
    const int in = net.w[l], out = net.w[l + 1];
    const int64_t n = (int64_t)in * out;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
      const int i = (int)(idx / out), o = (int)(idx - (int64_t)i * out);
      wt[net.offT[l] + idx] = theta[net.offW[l] + (int64_t)o * in + i];
    }
  }
}

__global__ void gpart_reduce_kernel(const double* __restrict__ gpart, int64_t warps, int64_t ldg, int64_t n,
                                    double* out, int accumulate) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t w = 0; w < warps; w++) s += gpart[w * ldg + a];
    out[a] = accumulate ? out[a] + s : s;
  }
}

template <int EQ, int MODE, bool XO>
cudaError_t launch_eq(const JetArgs& a, cudaStream_t st, int64_t* warps_used) {
  constexpr int D = Eq<EQ>::D, NF = Eq<EQ>::NF;
  constexpr int CR = JT<D>::CR;
  constexpr int CF = (MODE == MODE_RESIDUAL) ? CR : JT<D>::CF;
  const int64_t per_warp = jet_smem_doubles(a.net, CF, CR, NF) * (int64_t)sizeof(double);
  constexpr int64_t kSmemCap = 227 * 1024;   // the opt-in maximum per block
  // Few points (the Hilbert nodes, the wall and decay rows, the normalisation point): fewer warps
  // per block spread them over all SMs, so each SM's FP64 pipe serves fewer of them (512 nodes in
  // blocks of 8 warps would use 64 of the 152 SMs).  Each point is one warp's work whatever the
  // block size, so the rows do not change.
  static const int sms = [] {
    int dev = 0, v = 0;
    const bool ok = cudaGetDevice(&dev) == cudaSuccess &&
                    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0;
    return ok ? v : 152;
  }();
  int wpb = 8;
  const int64_t spread = (a.n + sms - 1) / sms;
  if (spread < wpb) wpb = spread < 1 ? 1 : (int)spread;
  while (wpb > 1 && per_warp * wpb > kSmemCap) wpb--;
  if (per_warp > kSmemCap) return cudaErrorInvalidValue;
  const size_t smem = (size_t)per_warp * wpb;
  // the opt-in limit is the same for every launch: handles stepped from several host
  // threads must not lower it under one another's launches
  cudaError_t err = cudaFuncSetAttribute(jet_kernel<EQ, MODE, XO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemCap);
  if (err != cudaSuccess) return err;
  int64_t blocks = (a.n + wpb - 1) / wpb;
  const int64_t cap = kJetMaxBlocks;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (warps_used) *warps_used = blocks * wpb;
  if (a.n == 0) return cudaSuccess;
  jet_kernel<EQ, MODE, XO><<<(unsigned)blocks, wpb * 32, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <int EQ, bool XO>
cudaError_t launch_map(const JetArgs& a, cudaStream_t st, int64_t* w) {
  switch (a.mode) {
    case MODE_RESIDUAL: return launch_eq<EQ, MODE_RESIDUAL, XO>(a, st, w);
    case MODE_JACOBIAN: return launch_eq<EQ, MODE_JACOBIAN, XO>(a, st, w);
    default: return launch_eq<EQ, MODE_GRADIENT, XO>(a, st, w);
  }
}

template <int EQ>
cudaError_t launch_mode(const JetArgs& a, cudaStream_t st, int64_t* w) {
  return a.net.exp_out ? launch_map<EQ, true>(a, st, w) : launch_map<EQ, false>(a, st, w);
}

}  // namespace

cudaError_t launch_jet(const JetArgs& a, cudaStream_t st, int64_t* warps_used) {
  switch (a.eq) {
    case GN_BURGERS: return launch_mode<GN_BURGERS>(a, st, warps_used);
    case GN_CCF: return launch_mode<GN_CCF>(a, st, warps_used);
    case GN_IPM: return launch_mode<GN_IPM>(a, st, warps_used);
    case GN_BOUSSINESQ: return launch_mode<GN_BOUSSINESQ>(a, st, warps_used);
    default: return cudaErrorInvalidValue;
  }
}

int jet_gpart_warps(const NetDesc& net, int d, int nf, int64_t n_max) {
  (void)net; (void)d; (void)nf; (void)n_max;
  return kJetMaxBlocks * 8;  // upper bound of blocks * warps per block used by launch_eq
}

cudaError_t launch_transpose_weights(const NetDesc& net, const double* theta, double* wt, cudaStream_t st) {
  transpose_weights_kernel<<<64, 256, 0, st>>>(net, theta, wt);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_gpart_reduce(const double* gpart, int64_t warps, int64_t ldg, int64_t n, double* out,
                                int accumulate, cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  gpart_reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(gpart, warps, ldg, n, out, accumulate);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gn
