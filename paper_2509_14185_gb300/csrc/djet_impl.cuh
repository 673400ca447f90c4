// Derivative-loss rows (Methods, "Training Loss": the d1 and d2 losses that flatten the
// residual between collocation points):
//   d1 rows  sqrt(2 c_d1 rho / (N_d1 N_E d))   d_{y_i} R_k            (i = 1..d)
//   d2 rows  sqrt(2 c_d2 rho / (N_d2 N_E d^2)) d_{y_i} d_{y_j} R_k    (every ordered pair i, j)
// point-major, then k, then i (then j), so that 1/2 |r~|^2 over these rows is
// c_d1 L_d1 + c_d2 L_d2.
//
// The residual operators are those of the d0 rows; their y-derivatives come from truncated
// multivariate Taylor series.  One warp per point, as in the d0 kernel:
//  1. forward: Taylor coefficients of every network activation in the network inputs
//     z = (q, beta) around z(y), to total degree O_y + 1 (O_y = the residual's own order in
//     y plus the loss order; the extra degree along q gives the lambda column, since lambda
//     enters the network only through q).  a = W h + b acts on each coefficient; tanh acts by
//     series composition, tanh(a_0 + d) = sum_k tanh^(k)(a_0) d^k / k! (Horner in d).
//  2. residual chain in dual numbers (lane 0: d/d lambda; lane 1 + f C_R + c: d/d of output
//     f's coefficient c; more directions than lanes take a second pass): the inputs' series in
//     y (q = u^(-a/2), beta = y_2 u^(-1/2), u = 1 + |y|^2, by binomial series), the network
//     series composed with them, the envelopes, the residual operator on series, and the
//     rows as coefficients of the residual series.
//  3. reverse, per row: the seeds pulled back through the layers; through tanh by the
//     transpose of multiplication by the series tanh'(a) = 1 - h h.
// CCF: the velocity is the discrete Hilbert operator differentiated in the collocation point
// (the d0 operator's derivative, node values held fixed): U(x) = sum_j K_j(x) g_j + D(x) g(x)
// with K_j, D rational in x; the K part enters as per-point series coefficients of
// sum_j K_j g_j (its lambda and parameter dependence added by the Hilbert contraction of each
// coefficient, row-scaled by the d row / d U_m seeds this kernel writes), the D part in the
// chain.  Exponential output maps, Fourier-feature networks and second stages are not
// supported for these rows (the host refuses them).
#pragma once

#include <cmath>

#include "gn_internal.cuh"

namespace gn {
namespace djet {

constexpr int64_t kDJetMaxBlocks = 152 * 2;

// ---- truncated Taylor series in D variables, total degree <= O ---------------------------
// Coefficients (Taylor, i.e. derivative / multi-index factorial) in graded order: 1D index a;
// 2D (a, b) (a the first variable's exponent) at (a + b)(a + b + 1)/2 + b.
__host__ __device__ constexpr int nmono(int D, int O) { return D == 1 ? O + 1 : (O + 1) * (O + 2) / 2; }
template <int D> __host__ __device__ constexpr int mi(int a, int b) {
  return D == 1 ? a : (a + b) * (a + b + 1) / 2 + b;
}

struct Dl {
  double v, d;
};
__device__ __forceinline__ Dl operator+(Dl a, Dl b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dl operator-(Dl a, Dl b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dl operator*(Dl a, Dl b) { return {a.v * b.v, fma(a.v, b.d, a.d * b.v)}; }
__device__ __forceinline__ Dl operator*(double s, Dl a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dl dz() { return {0.0, 0.0}; }
__device__ __forceinline__ Dl dc(double v) { return {v, 0.0}; }
__device__ __forceinline__ double sval(double x) { return x; }
__device__ __forceinline__ double sval(Dl x) { return x.v; }
__device__ __forceinline__ double mulacc(double z, double x, double y) { return fma(x, y, z); }
__device__ __forceinline__ Dl mulacc(Dl z, Dl x, Dl y) {
  return {fma(x.v, y.v, z.v), fma(x.v, y.d, fma(x.d, y.v, z.d))};
}
__device__ __forceinline__ Dl mulacc(Dl z, Dl x, double y) { return {fma(x.v, y, z.v), fma(x.d, y, z.d)}; }
__device__ __forceinline__ Dl mulacc(Dl z, double x, Dl y) { return {fma(x, y.v, z.v), fma(x, y.d, z.d)}; }
template <class T> __device__ __forceinline__ T szero();
template <> __device__ __forceinline__ double szero<double>() { return 0.0; }
template <> __device__ __forceinline__ Dl szero<Dl>() { return dz(); }

// z = x y, truncated to degree O (z must not alias x or y)
template <int D, int O, class T, class U, class V>
__device__ __forceinline__ void smul(const T* x, const U* y, V* z) {
  constexpr int N = nmono(D, O);
#pragma unroll
  for (int k = 0; k < N; k++) z[k] = szero<V>();
  if constexpr (D == 1) {
#pragma unroll
    for (int a1 = 0; a1 <= O; a1++)
#pragma unroll
      for (int a2 = 0; a2 <= O - a1; a2++) z[a1 + a2] = mulacc(z[a1 + a2], x[a1], y[a2]);
  } else {
#pragma unroll
    for (int g1 = 0; g1 <= O; g1++)
#pragma unroll
      for (int b1 = 0; b1 <= g1; b1++)
#pragma unroll
        for (int g2 = 0; g2 <= O - g1; g2++)
#pragma unroll
          for (int b2 = 0; b2 <= g2; b2++) {
            const int k = mi<2>(g1 - b1 + g2 - b2, b1 + b2);
            z[k] = mulacc(z[k], x[mi<2>(g1 - b1, b1)], y[mi<2>(g2 - b2, b2)]);
          }
  }
}
// y = d/dz_v x (degree O - 1, top degree zero)
template <int D, int O, class T>
__device__ __forceinline__ void sdiff(const T* x, int v, T* y) {
  constexpr int N = nmono(D, O);
#pragma unroll
  for (int k = 0; k < N; k++) y[k] = szero<T>();
  if constexpr (D == 1) {
#pragma unroll
    for (int a = 0; a < O; a++) y[a] = (double)(a + 1) * x[a + 1];
  } else {
#pragma unroll
    for (int g = 0; g < O; g++)
#pragma unroll
      for (int b = 0; b <= g; b++) {
        const int a = g - b;
        y[mi<2>(a, b)] = (v == 0) ? (double)(a + 1) * x[mi<2>(a + 1, b)] : (double)(b + 1) * x[mi<2>(a, b + 1)];
      }
  }
}
// (1 + w)^e for a series w with w_0 = 0 and a dual exponent e: sum_k binom(e, k) w^k (Horner)
template <int D, int O>
__device__ __forceinline__ void spow1p(const double* w, Dl e, Dl* out) {
  constexpr int N = nmono(D, O);
  Dl c[O + 1];
  c[0] = dc(1.0);
#pragma unroll
  for (int k = 1; k <= O; k++) c[k] = c[k - 1] * ((1.0 / k) * (e - dc((double)(k - 1))));
  Dl h[N], t[N];
#pragma unroll
  for (int k = 0; k < N; k++) h[k] = dz();
  h[0] = c[O];
#pragma unroll
  for (int k = O - 1; k >= 0; k--) {
    smul<D, O>(h, w, t);
#pragma unroll
    for (int q = 0; q < N; q++) h[q] = t[q];
    h[0] = h[0] + c[k];
  }
#pragma unroll
  for (int k = 0; k < N; k++) out[k] = h[k];
}
// tanh of a series (degree O): Horner in d = a - a_0 with the coefficients tanh^(k)(a_0) / k!,
// the derivatives from P_0 = T, P_{k+1}(T) = P_k'(T) (1 - T^2) (polynomials in T = tanh a_0)
template <int D, int O>
__device__ __forceinline__ void stanh(const double* a, double* h) {
  constexpr int N = nmono(D, O);
  const double T = tanh(a[0]);
  double ck[O + 1];
  double pc[O + 3];   // coefficients of P_k in T (degree k + 1)
#pragma unroll
  for (int i = 0; i < O + 3; i++) pc[i] = 0.0;
  pc[1] = 1.0;
  double fact = 1.0;
#pragma unroll
  for (int k = 0; k <= O; k++) {
    double v = 0.0;
#pragma unroll
    for (int i = O + 2; i >= 0; i--) v = fma(v, T, pc[i]);
    if (k > 0) fact *= k;
    ck[k] = v / fact;
    // P_{k+1} = P_k' (1 - T^2)
    double dp[O + 3];
#pragma unroll
    for (int i = 0; i < O + 3; i++) dp[i] = (i + 1 < O + 3) ? (i + 1) * pc[i + 1] : 0.0;
#pragma unroll
    for (int i = 0; i < O + 3; i++) pc[i] = dp[i] - ((i >= 2) ? dp[i - 2] : 0.0);
  }
  double d[N], t[N];
#pragma unroll
  for (int k = 0; k < N; k++) {
    d[k] = (k == 0) ? 0.0 : a[k];
    h[k] = 0.0;
  }
  h[0] = ck[O];
#pragma unroll
  for (int k = O - 1; k >= 0; k--) {
    smul<D, O>(h, d, t);
#pragma unroll
    for (int q = 0; q < N; q++) h[q] = t[q];
    h[0] += ck[k];
  }
}

template <int EQ> struct DEq;
template <> struct DEq<GN_BURGERS> { static constexpr int D = 1, NF = 1, NE = 1; };
template <> struct DEq<GN_CCF> { static constexpr int D = 1, NF = 1, NE = 1; };
template <> struct DEq<GN_IPM> { static constexpr int D = 2, NF = 2, NE = 2; };
template <> struct DEq<GN_BOUSSINESQ> { static constexpr int D = 2, NF = 3, NE = 3; };

// Orders of the row kind: the residual's own order in y (1 in 1D, 2 in 2D) plus the loss order.
template <int D, int ORD> struct DOrd {
  static constexpr int OY = (D == 1 ? 1 : 2) + ORD;     // degree of the field series
  static constexpr int CR = nmono(D, OY);               // reverse-pass coefficients
  static constexpr int CF = nmono(D, OY + 1);           // forward coefficients (lambda column)
  static constexpr int NR = D == 1 ? 1 : (ORD == 1 ? 2 : 4);   // rows per equation
};

__host__ __device__ inline int64_t djet_smem_doubles(const NetDesc& net, int CF, int CR, int NF) {
  const int64_t ldw = net.maxw;
  return (int64_t)net.L * CF * ldw + 2 * (int64_t)CR * ldw + (int64_t)NF * CF + 2;
}

template <int EQ, int ORD, int MODE>
__global__ void __launch_bounds__(256, 1) djet_kernel(const JetArgs A) {
  constexpr int D = DEq<EQ>::D, NF = DEq<EQ>::NF, NE = DEq<EQ>::NE;
  constexpr int OY = DOrd<D, ORD>::OY, CR = DOrd<D, ORD>::CR;
  constexpr int OF = (MODE == MODE_RESIDUAL) ? OY : OY + 1;
  constexpr int CF = nmono(D, OF);
  constexpr int NR = DOrd<D, ORD>::NR;
  constexpr int NROW = NE * NR;
  constexpr int K = 1 + NF * CR;                               // tangent directions
  constexpr int NPASS = (MODE == MODE_RESIDUAL) ? 1 : (K + 31) / 32;
  const NetDesc& net = A.net;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int ldw = net.maxw;
  const int L = net.L;
  extern __shared__ double sm[];
  double* H = sm + (int64_t)warp * djet_smem_doubles(net, DOrd<D, ORD>::CF, CR, NF);
  double* BA = H + (int64_t)L * CF * ldw;
  double* BB = BA + (int64_t)CR * ldw;
  double* NN = BB + (int64_t)CR * ldw;
  auto hc = [&](int j, int c) -> double* { return H + ((int64_t)j * CF + c) * ldw; };
  const int64_t gw = (int64_t)blockIdx.x * wpb + warp;
  const int64_t nw = (int64_t)gridDim.x * wpb;
  double* gp = (MODE == MODE_GRADIENT) ? A.gpart + gw * A.ldg : nullptr;
  const double lam = A.lamp ? *A.lamp : A.lam;

  for (int64_t pt = gw; pt < A.n; pt += nw) {
    double y[D];
#pragma unroll
    for (int k = 0; k < D; k++) y[k] = A.y[(int64_t)k * A.ystride + pt];
    double u0 = 1.0;
#pragma unroll
    for (int k = 0; k < D; k++) u0 = fma(y[k], y[k], u0);

    // ---- 1. network input series in (dq, dbeta) and the forward pass ------------------
    for (int idx = lane; idx < CF * ldw; idx += 32) H[idx] = 0.0;
    __syncwarp();
    const double a0 = 1.0 / (1.0 + lam);
    const double q0 = exp(-0.5 * a0 * log(u0));
    if (lane == 0) {
      hc(0, 0)[0] = q0;
      hc(0, mi<D>(1, 0))[0] = 1.0;
      if (D == 2) {
        hc(0, 0)[1] = y[D - 1] / sqrt(u0);
        hc(0, mi<D>(0, 1))[1] = 1.0;
      }
    }
    __syncwarp();
    for (int l = 0; l < L; l++) {
      const int in = net.w[l], out = net.w[l + 1];
      const double* wtl = A.wt + net.offT[l];
      const double* bl = A.theta + net.offB[l];
      for (int o = lane; o < out; o += 32) {
        double acc[CF];
        acc[0] = bl[o];
#pragma unroll
        for (int c = 1; c < CF; c++) acc[c] = 0.0;
        for (int i = 0; i < in; i++) {
          const double wv = __ldg(wtl + (int64_t)i * out + o);
#pragma unroll
          for (int c = 0; c < CF; c++) acc[c] = fma(wv, hc(l, c)[i], acc[c]);
        }
        if (l < L - 1) {
          double hs[CF];
          stanh<D, OF>(acc, hs);
#pragma unroll
          for (int c = 0; c < CF; c++) hc(l + 1, c)[o] = hs[c];
        } else {
#pragma unroll
          for (int c = 0; c < CF; c++) NN[o * CF + c] = acc[c];
        }
      }
      __syncwarp();
    }

    // ---- 2. residual chain in dual numbers, one or two passes over the directions ------
    const double w = A.wscale * (A.rho ? sqrt(A.rho[pt]) : 1.0);
    double rowv[NROW];
    double sd[NPASS][NROW];
    double sUv[ORD + 1];
#pragma unroll
    for (int e = 0; e < NROW; e++) rowv[e] = 0.0;
#pragma unroll
    for (int m = 0; m <= ORD; m++) sUv[m] = 0.0;
#pragma unroll
    for (int pass = 0; pass < NPASS; pass++) {
      const int dir = lane + 32 * pass;
      const bool ld = (dir == 0 && MODE != MODE_RESIDUAL);   // the lambda direction
      const Dl lamd = {lam, ld ? 1.0 : 0.0};
      const Dl a = {a0, ld ? -a0 * a0 : 0.0};
      // the network output coefficients along this direction (lambda: through q0 only)
      const double dq0 = -0.5 * log(u0) * q0 * a.d;             // d q0 / d lambda
      Dl nn[NF][CR];
#pragma unroll
      for (int f = 0; f < NF; f++)
#pragma unroll
        for (int c = 0; c < CR; c++) {
          double dv = 0.0;
          if (MODE != MODE_RESIDUAL) {
            if (ld) {
              // d c_alpha / d q0 = (alpha_q + 1) c_{alpha + e_q}
              int aq, ab;
              if (D == 1) { aq = c; ab = 0; }
              else { int g = 0; while ((g + 1) * (g + 2) / 2 <= c) g++; ab = c - g * (g + 1) / 2; aq = g - ab; }
              dv = (aq + 1) * NN[f * CF + mi<D>(aq + 1, ab)] * dq0;
            } else if (dir == 1 + f * CR + c) {
              dv = 1.0;
            }
          }
          nn[f][c] = {NN[f * CF + c], dv};
        }
      // u - u0 over u0 as a series in dy (exact, degree 2)
      double wsr[CR];
#pragma unroll
      for (int c = 0; c < CR; c++) wsr[c] = 0.0;
#pragma unroll
      for (int k = 0; k < D; k++) {
        const int e1 = (k == 0) ? mi<D>(1, 0) : mi<D>(0, 1);
        const int e2 = (k == 0) ? mi<D>(2, 0) : mi<D>(0, 2);
        wsr[e1] = 2.0 * y[k] / u0;
        wsr[e2] = 1.0 / u0;
      }
      // dq = q - q0 = q0 ((1 + w)^(-a/2) - 1), as a dual series; dbeta likewise (no lambda)
      Dl Pq[OY + 1][CR], Pb[D == 2 ? OY + 1 : 1][CR];
      {
        Dl t[CR];
        spow1p<D, OY>(wsr, (-0.5) * a, t);
        const Dl q0d = {q0, dq0};
#pragma unroll
        for (int c = 0; c < CR; c++) Pq[1][c] = (c == 0) ? dz() : q0d * t[c];
      }
      if constexpr (D == 2) {
        Dl t[CR];
        spow1p<D, OY>(wsr, dc(-0.5), t);
        // beta = (y2 + dy2) u0^(-1/2) (1 + w)^(-1/2)
        Dl ys[CR];
#pragma unroll
        for (int c = 0; c < CR; c++) ys[c] = dz();
        ys[0] = dc(y[1] / sqrt(u0));
        ys[mi<2>(0, 1)] = dc(1.0 / sqrt(u0));
        smul<D, OY>(ys, t, Pb[1]);
        Pb[1][0] = dz();
      }
      // powers
#pragma unroll
      for (int c = 0; c < CR; c++) Pq[0][c] = (c == 0) ? dc(1.0) : dz();
#pragma unroll
      for (int k = 2; k <= OY; k++) smul<D, OY>(Pq[k - 1], Pq[1], Pq[k]);
      if constexpr (D == 2) {
#pragma unroll
        for (int c = 0; c < CR; c++) Pb[0][c] = (c == 0) ? dc(1.0) : dz();
#pragma unroll
        for (int k = 2; k <= OY; k++) smul<D, OY>(Pb[k - 1], Pb[1], Pb[k]);
      }
      // network series composed with (dq, dbeta): G_f = sum_alpha nn_f[alpha] dq^a dbeta^b
      Dl G[NF][CR];
#pragma unroll
      for (int f = 0; f < NF; f++)
#pragma unroll
        for (int c = 0; c < CR; c++) G[f][c] = dz();
      if constexpr (D == 1) {
#pragma unroll
        for (int aq = 0; aq <= OY; aq++)
#pragma unroll
          for (int f = 0; f < NF; f++)
#pragma unroll
            for (int c = 0; c < CR; c++) G[f][c] = mulacc(G[f][c], nn[f][aq], Pq[aq][c]);
      } else {
#pragma unroll
        for (int g = 0; g <= OY; g++)
#pragma unroll
          for (int ab = 0; ab <= g; ab++) {
            const int aq = g - ab;
            Dl mono[CR];
            smul<D, OY>(Pq[aq], Pb[ab], mono);
#pragma unroll
            for (int f = 0; f < NF; f++)
#pragma unroll
              for (int c = 0; c < CR; c++) G[f][c] = mulacc(G[f][c], nn[f][mi<2>(aq, ab)], mono[c]);
          }
      }
      // envelopes y1^m u^e (e = e0 + k_f a / 2) times the network series
      auto envelope = [&](int m, Dl e, Dl* out) {
        Dl t[CR];
        spow1p<D, OY>(wsr, e, t);
        const double lu = log(u0);
        const double p = exp(e.v * lu);
        const Dl pe = {p, p * lu * e.d};                         // u0^e
        Dl ym[CR];
#pragma unroll
        for (int c = 0; c < CR; c++) ym[c] = dz();
        if (m == 0) ym[0] = dc(1.0);
        else if (m == 1) { ym[0] = dc(y[0]); ym[mi<D>(1, 0)] = dc(1.0); }
        else { ym[0] = dc(y[0] * y[0]); ym[mi<D>(1, 0)] = dc(2.0 * y[0]); ym[mi<D>(2, 0)] = dc(1.0); }
        Dl s[CR];
        smul<D, OY>(ym, t, s);
#pragma unroll
        for (int c = 0; c < CR; c++) out[c] = pe * s[c];
      };
      Dl F[NF][CR];
#pragma unroll
      for (int f = 0; f < NF; f++) {
        Dl kf;
        int m;
        double e0;
        if (EQ == GN_BURGERS) { kf = lamd; m = 1; e0 = -0.5; }
        else if (EQ == GN_CCF) { kf = lamd; m = 2; e0 = -1.0; }
        else if (EQ == GN_IPM) {
          if (f == 0) { kf = lamd; m = 0; e0 = 0.0; }
          else { kf = dc(1.0) + 2.0 * lamd; m = 1; e0 = -0.5; }
        } else {
          if (f == 0) { kf = dc(-1.0); m = 1; e0 = -0.5; }
          else if (f == 1) { kf = lamd + dc(-1.0); m = 0; e0 = 0.0; }
          else { kf = dc(1.0) + 2.0 * lamd; m = 1; e0 = -0.5; }
        }
        Dl env[CR];
        envelope(m, dc(e0) + 0.5 * (kf * a), env);
        smul<D, OY>(env, G[f], F[f]);
      }
      // residual series
      Dl R[NE][CR];
      const Dl opl = dc(1.0) + lamd;
      auto yser = [&](int k, Dl* out) {   // (1 + lambda) (y_k + dy_k)
#pragma unroll
        for (int c = 0; c < CR; c++) out[c] = dz();
        out[0] = y[k] * opl;
        out[(k == 0) ? mi<D>(1, 0) : mi<D>(0, 1)] = opl;
      };
      if constexpr (EQ == GN_BURGERS || EQ == GN_CCF) {
        Dl Uy[CR], V[CR], t[CR];
        sdiff<D, OY>(F[0], 0, Uy);
        yser(0, V);
        if constexpr (EQ == GN_BURGERS) {
#pragma unroll
          for (int c = 0; c < CR; c++) V[c] = V[c] + F[0][c];
        } else {
          // U = K part (series coefficients, lambda part added by the contraction) + D g
          Dl genv[CR], gs[CR], Ds[CR], Dg[CR];
          envelope(1, dc(-1.0) + 0.5 * (lamd * a), genv);
          smul<D, OY>(genv, G[0], gs);
#pragma unroll
          for (int c = 0; c < CR; c++) Ds[c] = dc(A.dcoef[(int64_t)c * A.n + pt]);
          smul<D, OY>(Ds, gs, Dg);
#pragma unroll
          for (int c = 0; c < CR; c++) V[c] = V[c] + Dg[c] + dc(A.ug[(int64_t)c * A.n + pt]);
          // d row / d U_m (the K part's coefficients): w ORD! [Theta']_{ORD - m}
#pragma unroll
          for (int m = 0; m <= ORD; m++) sUv[m] = w * (ORD == 2 ? 2.0 : 1.0) * Uy[ORD - m].v;
        }
        smul<D, OY>(V, Uy, t);
#pragma unroll
        for (int c = 0; c < CR; c++) R[0][c] = t[c] - lamd * F[0][c];
      } else {
        Dl d1[NF][CR], d2[NF][CR];
#pragma unroll
        for (int f = 0; f < NF; f++) {
          sdiff<D, OY>(F[f], 0, d1[f]);
          sdiff<D, OY>(F[f], 1, d2[f]);
        }
        constexpr int PS = NF - 1;   // the stream function is the last field
        Dl S11[CR], S22[CR];
        sdiff<D, OY>(d1[PS], 0, S11);
        sdiff<D, OY>(d2[PS], 1, S22);
        Dl V1[CR], V2[CR];
        yser(0, V1);
        yser(1, V2);
#pragma unroll
        for (int c = 0; c < CR; c++) {
          V1[c] = V1[c] + d2[PS][c];
          V2[c] = V2[c] - d1[PS][c];
        }
        Dl t1[CR], t2[CR];
        if constexpr (EQ == GN_IPM) {
          smul<D, OY>(V1, d1[0], t1);
          smul<D, OY>(V2, d2[0], t2);
#pragma unroll
          for (int c = 0; c < CR; c++) {
            R[0][c] = t1[c] + t2[c] - lamd * F[0][c];
            R[1][c] = S11[c] + S22[c] - d1[0][c];
          }
        } else {
          smul<D, OY>(V1, d1[0], t1);
          smul<D, OY>(V2, d2[0], t2);
#pragma unroll
          for (int c = 0; c < CR; c++) R[0][c] = F[0][c] + t1[c] + t2[c] - d1[1][c];
          smul<D, OY>(V1, d1[1], t1);
          smul<D, OY>(V2, d2[1], t2);
#pragma unroll
          for (int c = 0; c < CR; c++) R[1][c] = (dc(1.0) - lamd) * F[1][c] + t1[c] + t2[c];
#pragma unroll
          for (int c = 0; c < CR; c++) R[NE - 1][c] = S11[c] + S22[c] + F[0][c];
        }
      }
      // rows: d_i R_k (coefficient of e_i) or d_i d_j R_k (coefficient of e_i + e_j, times 2 if i == j)
#pragma unroll
      for (int k = 0; k < NE; k++)
#pragma unroll
        for (int r = 0; r < NR; r++) {
          Dl v;
          if (ORD == 1) {
            v = R[k][(r == 0) ? mi<D>(1, 0) : mi<D>(0, 1)];
          } else if (D == 1) {
            v = 2.0 * R[k][2];
          } else {
            const int i = r / 2, j = r % 2;
            v = (i == j) ? 2.0 * R[k][i == 0 ? mi<2>(2, 0) : mi<2>(0, 2)] : R[k][mi<2>(1, 1)];
          }
          if (pass == 0) rowv[k * NR + r] = w * v.v;
          sd[pass][k * NR + r] = w * v.d;
        }
    }

    // ---- 3. rows ---------------------------------------------------------------------
    const int64_t rbase = A.row0 + pt * NROW;
    if (lane == 0) {
#pragma unroll
      for (int e = 0; e < NROW; e++) {
        if (A.r) A.r[rbase + e] = rowv[e];
        if (!isfinite(rowv[e])) atomicOr(A.flag, 1);
      }
    }
    double comb[NROW];
    if (MODE == MODE_GRADIENT) {
#pragma unroll
      for (int e = 0; e < NROW; e++) comb[e] = A.seed ? A.seed[rbase + e] : rowv[e];
    }
    if (EQ == GN_CCF && A.sU && lane == 0) {
      const double cs = (MODE == MODE_GRADIENT) ? comb[0] : 1.0;
#pragma unroll
      for (int m = 0; m <= ORD; m++) A.sU[(int64_t)m * A.n + pt] = cs * sUv[m];
    }
    if (MODE == MODE_RESIDUAL) continue;

    const int nrev = (MODE == MODE_GRADIENT) ? 1 : NROW;
    for (int e = 0; e < nrev; e++) {
      const int64_t row = rbase + e;
      double* Jrow = nullptr;
      if (MODE == MODE_JACOBIAN) {
        if (row < A.jrow_lo || row >= A.jrow_hi) continue;
        Jrow = A.J + (row - A.jrow_lo) * A.ldJ;
      }
      double s[NPASS];
#pragma unroll
      for (int pass = 0; pass < NPASS; pass++) {
        if (MODE == MODE_GRADIENT) {
          double acc = 0.0;
#pragma unroll
          for (int ee = 0; ee < NROW; ee++) acc = fma(comb[ee], sd[pass][ee], acc);
          s[pass] = acc;
        } else {
          double v = 0.0;
#pragma unroll
          for (int ee = 0; ee < NROW; ee++)
            if (ee == e) v = sd[pass][ee];
          s[pass] = v;
        }
      }
      if (lane == 0) {   // the lambda column (zero while lambda is held fixed)
        if (MODE == MODE_JACOBIAN) Jrow[net.P] = A.lam_frozen ? 0.0 : s[0];
        else if (!A.lam_frozen) gp[net.P] += s[0];
      }
#pragma unroll
      for (int pass = 0; pass < NPASS; pass++) {
        const int dir = lane + 32 * pass;
        if (dir >= 1 && dir < K) {
          const int f = (dir - 1) / CR, c = (dir - 1) % CR;
          BA[c * ldw + f] = s[pass];
        }
      }
      __syncwarp();
      double* ab = BA;
      double* hb = BB;
      for (int l = L - 1; l >= 0; l--) {
        const int in = net.w[l], out = net.w[l + 1];
        const int64_t nW = (int64_t)out * in;
        const int64_t off = net.offW[l];
        for (int64_t idx = lane; idx < nW + out; idx += 32) {
          double v;
          if (idx < nW) {
            const int o = (int)(idx / in);
            const int i = (int)(idx - (int64_t)o * in);
            v = 0.0;
#pragma unroll
            for (int c = 0; c < CR; c++) v = fma(ab[c * ldw + o], hc(l, c)[i], v);
          } else {
            v = ab[idx - nW];
          }
          if (MODE == MODE_JACOBIAN) Jrow[off + idx] = v;
          else gp[off + idx] += v;
        }
        if (l == 0) break;
        const double* Wl = A.theta + off;
        for (int i = lane; i < in; i += 32) {
          double hbar[CR];
#pragma unroll
          for (int c = 0; c < CR; c++) hbar[c] = 0.0;
          for (int o = 0; o < out; o++) {
            const double wv = __ldg(Wl + (int64_t)o * in + i);
#pragma unroll
            for (int c = 0; c < CR; c++) hbar[c] = fma(wv, ab[c * ldw + o], hbar[c]);
          }
          // through h = tanh(a): a-bar_beta = sum_gamma h-bar_{beta + gamma} s_gamma, s = 1 - h h
          double hs[CR], sq[CR], sgm[CR];
#pragma unroll
          for (int c = 0; c < CR; c++) hs[c] = hc(l, c)[i];
          smul<D, OY>(hs, hs, sq);
#pragma unroll
          for (int c = 0; c < CR; c++) sgm[c] = (c == 0 ? 1.0 : 0.0) - sq[c];
          double abar[CR];
#pragma unroll
          for (int c = 0; c < CR; c++) abar[c] = 0.0;
          if constexpr (D == 1) {
#pragma unroll
            for (int b = 0; b <= OY; b++)
#pragma unroll
              for (int g = 0; g <= OY - b; g++) abar[b] = fma(hbar[b + g], sgm[g], abar[b]);
          } else {
#pragma unroll
            for (int g1 = 0; g1 <= OY; g1++)
#pragma unroll
              for (int b1 = 0; b1 <= g1; b1++)
#pragma unroll
                for (int g2 = 0; g2 <= OY - g1; g2++)
#pragma unroll
                  for (int b2 = 0; b2 <= g2; b2++) {
                    const int kb = mi<2>(g1 - b1, b1), kg = mi<2>(g2 - b2, b2);
                    const int ks = mi<2>(g1 - b1 + g2 - b2, b1 + b2);
                    abar[kb] = fma(hbar[ks], sgm[kg], abar[kb]);
                  }
          }
#pragma unroll
          for (int c = 0; c < CR; c++) hb[c * ldw + i] = abar[c];
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

template <int EQ, int ORD, int MODE>
cudaError_t launch_ord(const JetArgs& a, cudaStream_t st, int64_t* warps_used) {
  constexpr int D = DEq<EQ>::D, NF = DEq<EQ>::NF;
  const int64_t per_warp =
      djet_smem_doubles(a.net, DOrd<D, ORD>::CF, DOrd<D, ORD>::CR, NF) * (int64_t)sizeof(double);
  constexpr int64_t kSmemCap = 227 * 1024;
  int wpb = 8;
  while (wpb > 1 && per_warp * wpb > kSmemCap) wpb--;
  if (per_warp > kSmemCap) return cudaErrorInvalidValue;
  cudaError_t err = cudaFuncSetAttribute(djet_kernel<EQ, ORD, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemCap);
  if (err != cudaSuccess) return err;
  int64_t blocks = (a.n + wpb - 1) / wpb;
  if (blocks > kDJetMaxBlocks) blocks = kDJetMaxBlocks;
  if (blocks < 1) blocks = 1;
  if (warps_used) *warps_used = blocks * wpb;
  if (a.n == 0) return cudaSuccess;
  djet_kernel<EQ, ORD, MODE><<<(unsigned)blocks, wpb * 32, (size_t)per_warp * wpb, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <int EQ, int ORD>
cudaError_t launch_mode(const JetArgs& a, cudaStream_t st, int64_t* w) {
  switch (a.mode) {
    case MODE_RESIDUAL: return launch_ord<EQ, ORD, MODE_RESIDUAL>(a, st, w);
    case MODE_JACOBIAN: return launch_ord<EQ, ORD, MODE_JACOBIAN>(a, st, w);
    default: return launch_ord<EQ, ORD, MODE_GRADIENT>(a, st, w);
  }
}

template <int EQ>
cudaError_t launch_eq(const JetArgs& a, int ord, cudaStream_t st, int64_t* w) {
  return ord == 1 ? launch_mode<EQ, 1>(a, st, w) : launch_mode<EQ, 2>(a, st, w);
}

}  // namespace djet
}  // namespace gn
