"""Self-similar profile problems: ansatz, network and residual operators (FP64).

Paper, Methods, "Self-similar Solutions": phi_A(x, t) = (1-t)^{k_A(lambda)} Phi_A(y),
y = x / (1-t)^{1+lambda}; substituting into each PDE and factoring out the
power of (1-t) gives the static equations E_k(Phi, lambda) = 0 (Eq.
self-similar-static).  With tau = 1 - t, a time derivative of tau^k Phi(y)
is tau^{k-1} [-k Phi + (1+lambda) y . grad Phi]; velocities scale as
tau^lambda.  V = (1+lambda) y + U denotes the self-similar transport velocity.
The resulting residual operators (this project's derivation; the paper's own
are in its Supplementary Information):

  Burgers      u_t + u u_x = 0            k_u = lambda
               R = -lambda U + ((1+lambda) y + U) U'
  CCF          theta_t + (H theta) theta_x = 0     k = lambda, U = H Theta
               R = -lambda Theta + ((1+lambda) y + U) Theta'
  IPM          rho_t + u . grad rho = 0, Delta psi = d1 rho, u = (d2 psi, -d1 psi)
               k_rho = lambda, k_psi = 1 + 2 lambda
               R1 = -lambda P + V . grad P,   R2 = Delta Psi - d1 P
  Boussinesq   omega_t + u . grad omega = d1 theta, theta_t + u . grad theta = 0,
               -Delta psi = omega, u = (d2 psi, -d1 psi)
               k_omega = -1, k_theta = lambda - 1, k_psi = 1 + 2 lambda
               R_Omega = Omega + V . grad Omega - d1 Theta
               R_Theta = (1 - lambda) Theta + V . grad Theta
               R_Psi   = Delta Psi + Omega
In the Boussinesq case d11 R_Theta at the origin reproduces the paper's printed
lambda-inference rule lambda = -3 - 2 d1 U1(0, 0) (Methods, "Identifying
admissible lambda values", item 2); a test checks this symbolically.

Ansatz (Methods, "Solution Modeling", Eq. ansatz_vorticity and its stated
generalisation to every field): Phi_A(y) = s_A(y) * NN_A(z(y)) * q^{-k_A},
with q = (1 + |y|^2)^{-1/(2(1+lambda))}, beta = y2 / sqrt(1 + |y|^2),
z = q (1D) or (q, beta) (2D), s_A = y1 / sqrt(1+|y|^2) for odd fields and
1 for even fields (CCF Theta: y^2 / (1+y^2), which removes the forced zero
at the origin).  For Omega (k = -1) this is exactly Eq. ansatz_vorticity.
NN is a tanh MLP with a linear output layer; theta stores, per layer, W
(out x in, row-major) then b.
"""
from __future__ import annotations

import numpy as np

from . import hilbert
from .jets import Jet
from .taylor import Taylor

BURGERS, CCF, IPM, BOUSSINESQ = 0, 1, 2, 3
DIM = {BURGERS: 1, CCF: 1, IPM: 2, BOUSSINESQ: 2}
N_EQ = {BURGERS: 1, CCF: 1, IPM: 2, BOUSSINESQ: 3}
N_FIELDS = {BURGERS: 1, CCF: 1, IPM: 2, BOUSSINESQ: 3}
HAS_WALL = {BURGERS: False, CCF: False, IPM: True, BOUSSINESQ: True}


# ---------------------------------------------------------------------------
# residual operators on field values and derivatives (plain arithmetic, so
# they also accept sympy expressions)
# ---------------------------------------------------------------------------

def residual_burgers(lam, y, U, U_y):
    return [-lam * U + ((1 + lam) * y + U) * U_y]


def residual_ccf(lam, y, Th, Th_y, Uvel):
    return [-lam * Th + ((1 + lam) * y + Uvel) * Th_y]


def residual_ipm(lam, y1, y2, P, P_1, P_2, Psi_1, Psi_2, Psi_11, Psi_22):
    U1, U2 = Psi_2, -Psi_1
    V1, V2 = (1 + lam) * y1 + U1, (1 + lam) * y2 + U2
    return [-lam * P + V1 * P_1 + V2 * P_2,
            Psi_11 + Psi_22 - P_1]


def residual_boussinesq(lam, y1, y2, Om, Om_1, Om_2, Th, Th_1, Th_2, Psi_1, Psi_2, Psi_11, Psi_22):
    U1, U2 = Psi_2, -Psi_1
    V1, V2 = (1 + lam) * y1 + U1, (1 + lam) * y2 + U2
    return [Om + V1 * Om_1 + V2 * Om_2 - Th_1,
            (1 - lam) * Th + V1 * Th_1 + V2 * Th_2,
            Psi_11 + Psi_22 + Om]


# Exponent k_A(lambda) and prefactor kind of every field, in network-output order.
# prefactor: "odd" = y1/sqrt(u), "even" = 1, "ccf" = y^2/u, "g" = y/u.
def field_specs(eq, lam):
    if eq == BURGERS:
        return [("odd", lam)]
    if eq == CCF:
        return [("ccf", lam)]
    if eq == IPM:
        return [("even", lam), ("odd", 1 + 2 * lam)]
    if eq == BOUSSINESQ:
        return [("odd", -1.0 + 0 * lam), ("even", lam - 1), ("odd", 1 + 2 * lam)]
    raise ValueError(eq)


def _prefactor(kind, ys, u):
    y1 = ys[0]
    if kind == "odd":
        return y1 / u.sqrt()
    if kind == "even":
        return y1.ones_like()
    if kind == "ccf":
        return (y1 * y1) / u
    if kind == "g":
        return y1 / u
    raise ValueError(kind)


class Problem:
    """One profile fit: equation, MLP widths, collocation and wall points, loss weights."""

    def __init__(self, equation, widths, y, y_bnd=None, rho=None, c_bnd=1.0,
                 y_norm=(1.0, 0.0), c_norm=1.0, c_norm_w=1.0, hilbert_m=1024, stage1=None, fourier=None,
                 y_inf=None, c_inf=1.0, norm_field=None, norm_deriv=None, output_map=0,
                 y_d1=None, rho_d1=None, c_d1=1.0, y_d2=None, rho_d2=None, c_d2=1.0,
                 y_relu=None, c_relu=1.0, relu_bound=0.0, relu_sign=1):
        self.eq = int(equation)
        self.widths = list(widths)
        self.d = DIM[self.eq]
        assert self.widths[0] == self.d and self.widths[-1] == N_FIELDS[self.eq]
        self.y = np.asarray(y, dtype=np.float64).reshape(self.d, -1)
        self.n = self.y.shape[1]
        if y_bnd is None or not HAS_WALL[self.eq]:
            self.y_bnd = np.zeros((self.d, 0))
        else:
            self.y_bnd = np.asarray(y_bnd, dtype=np.float64).reshape(self.d, -1)
        self.nb = self.y_bnd.shape[1]
        self.rho = np.ones(self.n) if rho is None else np.asarray(rho, dtype=np.float64)
        self.c_bnd = float(c_bnd)
        self.y_norm = tuple(float(v) for v in y_norm)
        self.c_norm = float(c_norm)
        self.c_norm_w = float(c_norm_w)
        # the constrained field A0 and whether the normalisation row takes its value (0) or its
        # d/dy1 (1) (Methods, "Training Loss": constraints on a field's values or derivatives).
        # Defaults: field 0's value, except Boussinesq's d1 Omega(0, 0) = 1
        self.norm_field = 0 if norm_field is None else int(norm_field)
        self.norm_deriv = (1 if self.eq == BOUSSINESQ else 0) if norm_deriv is None else int(norm_deriv)
        assert 0 <= self.norm_field < N_FIELDS[self.eq] and self.norm_deriv in (0, 1)
        # decay points Y_inf of the data loss (Methods, "Training Loss", second data-loss term):
        # the normalised field must vanish far from the origin
        self.y_inf = (np.zeros((self.d, 0)) if y_inf is None
                      else np.asarray(y_inf, dtype=np.float64).reshape(self.d, -1))
        self.ninf = self.y_inf.shape[1]
        self.c_inf = float(c_inf)
        # derivative losses (Methods, "Training Loss", d1 and d2): batches Y1, Y2 with per-point
        # weights rho and loss coefficients c_d1, c_d2
        self.y_d1 = np.zeros((self.d, 0)) if y_d1 is None else np.asarray(y_d1, np.float64).reshape(self.d, -1)
        self.y_d2 = np.zeros((self.d, 0)) if y_d2 is None else np.asarray(y_d2, np.float64).reshape(self.d, -1)
        self.n_d1, self.n_d2 = self.y_d1.shape[1], self.y_d2.shape[1]
        self.rho_d1 = np.ones(self.n_d1) if rho_d1 is None else np.asarray(rho_d1, np.float64)
        self.rho_d2 = np.ones(self.n_d2) if rho_d2 is None else np.asarray(rho_d2, np.float64)
        self.c_d1, self.c_d2 = float(c_d1), float(c_d2)
        # bound constraints of the data loss (Methods, "Training Loss": a constraint acted on by
        # a relu before squaring): relu(s (Phi_A0(y) - b)) at the points, s = +1 an upper bound
        # b on the constrained field, s = -1 a lower bound
        self.y_relu = np.zeros((self.d, 0)) if y_relu is None else np.asarray(y_relu, np.float64).reshape(self.d, -1)
        self.nrelu = self.y_relu.shape[1]
        self.c_relu, self.relu_bound, self.relu_sign = float(c_relu), float(relu_bound), int(relu_sign)
        assert self.relu_sign in (1, -1)
        self.M = int(hilbert_m)
        self.ne = N_EQ[self.eq]
        # last activation of the network (Methods, "Solution Modeling": exponential or
        # exponential-adjacent): 0 linear (the default reading), 1 exp; a stage-1 network of a
        # stage-2 problem uses the same map
        self.output_map = int(output_map)
        assert self.output_map in (0, 1)
        # Fourier-feature network (Methods, "Multi-stage Training", item 2): fourier = B, an
        # (m' x m) array drawn by the caller; the layer after the linear input layer (widths[1]
        # = m) is the fixed map x -> [cos(B x), sin(B x)] (widths[2] = 2 m'), not trained.
        self.fourier = None if fourier is None else np.asarray(fourier, dtype=np.float64)
        if self.fourier is not None:
            assert self.fourier.shape == (self.widths[2] // 2, self.widths[1]) and self.widths[2] % 2 == 0
        self.P = sum(self.widths[i] * self.widths[i + 1] + self.widths[i + 1]
                     for i in range(len(self.widths) - 1) if not (self.fourier is not None and i == 1))
        self.n_rows = (self.n * self.ne + self.n_d1 * self.ne * self.d + self.n_d2 * self.ne * self.d ** 2
                       + self.nb + self.ninf + self.nrelu + 1)
        # Multi-stage training (Methods, "Multi-stage Training"): stage1 = (widths1, theta1, eps)
        # makes every field Phi = Phi_1 + eps Phi_2 with Phi_1 the frozen stage-1 network and
        # Phi_2 this problem's network, and divides every row by eps (the normalised stage-2
        # equation: R(Phi_1 + eps Phi_2) / eps = R_1 / eps + D[Phi_1] Phi_2 + O(eps)).
        self.stage1 = None
        if stage1 is not None:
            w1, th1, eps = stage1
            w1 = list(w1)
            assert w1[0] == self.d and w1[-1] == N_FIELDS[self.eq] and eps > 0
            self.stage1 = (w1, np.asarray(th1, dtype=np.float64), float(eps))

    # -- network ----------------------------------------------------------
    def layers(self, theta, widths=None, fourier=None):
        """(W, b) per layer from theta; with a Fourier layer its entry is (B, None), not in theta."""
        widths = self.widths if widths is None else widths
        out, off = [], 0
        for i in range(len(widths) - 1):
            fi, fo = widths[i], widths[i + 1]
            if fourier is not None and i == 1:
                out.append((fourier, None))
                continue
            W = theta[off:off + fi * fo].reshape(fo, fi)
            off += fi * fo
            b = theta[off:off + fo]
            off += fo
            out.append((W, b))
        assert off == len(theta)
        return out

    def mlp(self, theta, z, widths=None, fourier=None):
        """tanh MLP with a linear (or, with output_map = 1, exponential) last layer applied to
        the input jet z (components (d_in, n)).  With a Fourier layer: linear input layer (no
        activation), then [cos(B x), sin(B x)]."""
        h = z
        L = self.layers(theta, widths, fourier)
        for i, (W, b) in enumerate(L):
            a = h.matvec(W, b)
            if i == len(L) - 1:
                h = a.exp() if self.output_map == 1 else a
            elif fourier is not None and i == 0:
                h = a
            elif fourier is not None and i == 1:
                h = type(a).vconcat(a.cos(), a.sin())
            else:
                h = a.tanh()
        return h

    # -- ansatz -------------------------------------------------------------
    def fields(self, theta, lam, ys, extra_g=False, order=None):
        """Field jets Phi_A at points ys (d, n); for CCF optionally also g = Theta / y.
        In a stage-2 problem: Phi_1 + eps Phi_2 (and g_1 + eps g_2).  order: None for the
        second-order Jet, else truncated Taylor series of that total order in y."""
        out = self.network_fields(theta, lam, ys, extra_g, order=order)
        if self.stage1 is None:
            return out
        w1, th1, eps = self.stage1
        base = self.network_fields(th1, lam, ys, extra_g, widths=w1, order=order)
        return [b + f * eps for b, f in zip(base, out)]

    def network_fields(self, theta, lam, ys, extra_g=False, widths=None, order=None):
        """The ansatz fields of one network (widths, theta) at points ys (second-order jets,
        or Taylor series of the given order in y)."""
        d = self.d
        if order is None:
            yj = [Jet.variable(ys[i], i, d) for i in range(d)]
            u = Jet.const(np.ones(ys.shape[1]), d)
        else:
            yj = [Taylor.variable(ys[i], i, d, order) for i in range(d)]
            u = Taylor.const(np.ones(ys.shape[1]), d, order, like=ys[0])
        for i in range(d):
            u = u + yj[i] * yj[i]
        q = u.pow(-1.0 / (2.0 * (1.0 + lam)))
        if d == 1:
            z = type(q).stack([q])
        else:
            beta = yj[1] / u.sqrt()
            z = type(q).stack([q, beta])
        nn = self.mlp(theta, z, widths, self.fourier if widths is None else None)
        out = []
        for a, (kind, k) in enumerate(field_specs(self.eq, lam)):
            out.append(_prefactor(kind, yj, u) * nn[a] * q.pow(-k))
        if extra_g:
            k = field_specs(self.eq, lam)[0][1]
            out.append(_prefactor("g", yj, u) * nn[0] * q.pow(-k))
        return out

    def interior_residuals(self, theta, lam, ys=None):
        ys = self.y if ys is None else ys
        if self.eq == BURGERS:
            (U,) = self.fields(theta, lam, ys)
            return residual_burgers(lam, ys[0], U.v, U.g[0])
        if self.eq == CCF:
            Th, g = self.fields(theta, lam, ys, extra_g=True)
            _, s = hilbert.nodes(self.M)
            g_nodes = self.fields(theta, lam, s.reshape(1, -1), extra_g=True)[1].v
            Uvel = hilbert.velocity(ys[0], g.v, g_nodes, self.M)
            return residual_ccf(lam, ys[0], Th.v, Th.g[0], Uvel)
        if self.eq == IPM:
            P, Psi = self.fields(theta, lam, ys)
            return residual_ipm(lam, ys[0], ys[1], P.v, P.g[0], P.g[1],
                                Psi.g[0], Psi.g[1], Psi.h[0][0], Psi.h[1][1])
        if self.eq == BOUSSINESQ:
            Om, Th, Psi = self.fields(theta, lam, ys)
            return residual_boussinesq(lam, ys[0], ys[1], Om.v, Om.g[0], Om.g[1],
                                       Th.v, Th.g[0], Th.g[1], Psi.g[0], Psi.g[1],
                                       Psi.h[0][0], Psi.h[1][1])
        raise ValueError(self.eq)

    def residual_series(self, theta, lam, ys, order):
        """The residuals R_k at the points ys as Taylor series in y: the operators applied to
        the fields' series of the given total order (the residuals lose one order per
        derivative they take: one in 1D, two in 2D).  For CCF the velocity is the discrete
        Hilbert operator differentiated in the collocation point (the paper leaves its
        derivative undefined; this is the derivative of the operator the d0 residual uses)."""
        d = self.d
        Y = [Taylor.variable(ys[i], i, d, order) for i in range(d)]
        if self.eq == BURGERS:
            (U,) = self.fields(theta, lam, ys, order=order)
            return residual_burgers(lam, Y[0], U, U.diff(0))
        if self.eq == IPM:
            P, Psi = self.fields(theta, lam, ys, order=order)
            return residual_ipm(lam, Y[0], Y[1], P, P.diff(0), P.diff(1), Psi.diff(0), Psi.diff(1),
                                Psi.diff(0).diff(0), Psi.diff(1).diff(1))
        if self.eq == BOUSSINESQ:
            Om, Th, Psi = self.fields(theta, lam, ys, order=order)
            return residual_boussinesq(lam, Y[0], Y[1], Om, Om.diff(0), Om.diff(1), Th, Th.diff(0), Th.diff(1),
                                       Psi.diff(0), Psi.diff(1), Psi.diff(0).diff(0), Psi.diff(1).diff(1))
        if self.eq == CCF:
            # the discrete velocity differentiated in the collocation point (the node values
            # do not move): the derivative of the operator that defines the d0 residual
            Th, g = self.fields(theta, lam, ys, extra_g=True, order=order)
            _, s = hilbert.nodes(self.M)
            g_nodes = self.fields(theta, lam, s.reshape(1, -1), extra_g=True)[1].v
            Uvel = hilbert.velocity_series(Y[0], g, g_nodes, self.M)
            return residual_ccf(lam, Y[0], Th, Th.diff(0), Uvel)
        raise ValueError(self.eq)

    def d1_residuals(self, theta, lam, ys=None):
        """d R_k / d y_i at the points: array (N_E, d, n)."""
        ys = self.y_d1 if ys is None else ys
        Rs = self.residual_series(theta, lam, ys, 3)
        return np.array([[R.diff(i).v for i in range(self.d)] for R in Rs])

    def d2_residuals(self, theta, lam, ys=None):
        """d^2 R_k / d y_i d y_j at the points, every ordered pair (i, j): array (N_E, d, d, n)."""
        ys = self.y_d2 if ys is None else ys
        Rs = self.residual_series(theta, lam, ys, 4)
        return np.array([[[R.diff(i).diff(j).v for j in range(self.d)] for i in range(self.d)] for R in Rs])

    def wall_values(self, theta, lam):
        """No-penetration on the wall y2 = 0: the stream function vanishes there."""
        if self.nb == 0:
            return np.zeros(0)
        return self.fields(theta, lam, self.y_bnd)[-1].v

    def inf_values(self, theta, lam):
        """Decay constraint values Phi_{A0}(y) at the points of Y_inf: the value (not a
        derivative) of the normalised field A0."""
        if self.ninf == 0:
            return np.zeros(0)
        return self.fields(theta, lam, self.y_inf)[self.norm_field].v

    def relu_values(self, theta, lam):
        """relu(s (Phi_A0(y) - b)) at the bound points; the relu decides on the real part, so a
        complex step passes through active rows and vanishes on inactive ones."""
        if self.nrelu == 0:
            return np.zeros(0)
        x = self.relu_sign * (self.fields(theta, lam, self.y_relu)[self.norm_field].v - self.relu_bound)
        return np.where(np.real(x) > 0.0, x, 0.0 * x)

    def norm_value(self, theta, lam):
        """Normalisation constraint value Phi_{A0}(y_norm), or its d/dy1 (the Boussinesq
        default: d1 Omega there)."""
        ys = np.array(self.y_norm[:self.d], dtype=np.float64).reshape(self.d, 1)
        F = self.fields(theta, lam, ys)[self.norm_field]
        if self.norm_deriv:
            return F.g[0][0]
        return F.v[0]

    # -- weighted rows ------------------------------------------------------
    def rows(self, theta, lam):
        """r~ such that h = 1/2 |r~|^2 is the paper's equation loss plus data loss:
        h = (1/(N N_E)) sum rho R^2 + c_d1 L_d1 + c_d2 L_d2 + (c_bnd/N_b) sum R_b^2
            + c_inf sum_{Y_inf} Phi(y)^2 + c_relu sum relu(s (Phi(y) - b))^2 + c_norm_w (Phi(y_norm) - C)^2
        (rows in that order: interior point-major, d1, d2, wall, decay, bounds, normalisation last)."""
        R = self.interior_residuals(theta, lam)
        w = np.sqrt(2.0 * self.rho / (self.n * self.ne))
        inner = np.stack([w * Rk for Rk in R], axis=1).reshape(-1)   # point-major
        parts = [inner]
        # derivative losses: c_d1 / (N_d1 N_E d) sum rho (d_i R_k)^2 and c_d2 / (N_d2 N_E d^2) sum
        # rho (d_i d_j R_k)^2, rows point-major, then k, then i (and j)
        if self.n_d1:
            D1 = self.d1_residuals(theta, lam)                   # (ne, d, n)
            w1 = np.sqrt(2.0 * self.c_d1 * self.rho_d1 / (self.n_d1 * self.ne * self.d))
            parts.append((np.moveaxis(D1, -1, 0) * w1[:, None, None]).reshape(-1))
        if self.n_d2:
            D2 = self.d2_residuals(theta, lam)                   # (ne, d, d, n)
            w2 = np.sqrt(2.0 * self.c_d2 * self.rho_d2 / (self.n_d2 * self.ne * self.d ** 2))
            parts.append((np.moveaxis(D2, -1, 0) * w2[:, None, None, None]).reshape(-1))
        if self.nb:
            parts.append(np.sqrt(2.0 * self.c_bnd / self.nb) * self.wall_values(theta, lam))
        if self.ninf:
            parts.append(np.sqrt(2.0 * self.c_inf) * self.inf_values(theta, lam))
        if self.nrelu:
            parts.append(np.sqrt(2.0 * self.c_relu) * self.relu_values(theta, lam))
        parts.append(np.array([np.sqrt(2.0 * self.c_norm_w) * (self.norm_value(theta, lam) - self.c_norm)]))
        r = np.concatenate(parts)
        return r / self.stage1[2] if self.stage1 is not None else r

    def loss(self, theta, lam):
        r = self.rows(theta, lam)
        return 0.5 * float(np.dot(r, r))

    def max_abs_residual(self, theta, lam, ys=None):
        """Max d0 residual over a grid (Methods, "Validation Metrics", max d0 residual)."""
        R = self.interior_residuals(theta, lam, ys)
        return float(max(np.max(np.abs(Rk)) for Rk in R))
