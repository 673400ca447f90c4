"""Discrete Hilbert operator for the CCF velocity u = H theta.

The paper names the CCF model (theta_t + (H theta) theta_x = 0) but gives
neither the equation nor its discretisation (both deferred to the
Supplementary Information).  This project's reading, written out here as a
plain sum:

  H f(x) = (1/pi) p.v. int f(s) / (x - s) ds.

Theta grows like |y|^(lambda/(1+lambda)), so write Theta(s) = s * g(s) with
g odd and decaying; then H Theta(x) = x * H g(x) because int g = 0.
With s = tan(psi/2), x = tan(phi/2) one has
  ds / (x - s) = (1/2) [cot((phi - psi)/2) - tan(psi/2)] dpsi,
so H g(x) = C[G](phi) - c0 with G(psi) = g(tan(psi/2)),
  C[G](phi) = (1/2pi) p.v. int G(psi) cot((phi - psi)/2) dpsi  (periodic
  conjugate function), c0 = (1/2pi) int G(psi) tan(psi/2) dpsi.
Both integrals are taken by the M-point trapezoid rule on the nodes
psi_j = -pi + (j + 1/2) 2pi/M, and the principal value by subtracting
G(phi) (the periodic cot kernel integrates to zero):
  U(x) = x * [ (1/M) sum_j (g_j - g(x)) cot((phi - psi_j)/2)
               - (1/M) sum_j g_j tan(psi_j/2) ].
This discrete operator *defines* the CCF residual for parity purposes.
"""
from __future__ import annotations

import numpy as np


def nodes(M: int):
    """Circle nodes psi_j and their images s_j = tan(psi_j / 2) on the real line."""
    j = np.arange(M, dtype=np.float64)
    psi = -np.pi + (j + 0.5) * (2.0 * np.pi / M)
    return psi, np.tan(0.5 * psi)


def velocity(x, g_at_x, g_nodes, M: int):
    """U(x) = x * H g(x) by the singularity-subtracted trapezoid rule above.

    x: (n,) real collocation points; g_at_x: (n,) values g(x); g_nodes: (M,)
    values g(s_j).  g may be complex (complex-step differentiation)."""
    psi, s = nodes(M)
    phi = 2.0 * np.arctan(np.asarray(x, dtype=np.float64))
    cot = 1.0 / np.tan(0.5 * (phi[:, None] - psi[None, :]))           # (n, M)
    conj = ((g_nodes[None, :] - g_at_x[:, None]) * cot).sum(axis=1) / M
    c0 = (g_nodes * s).sum() / M
    return x * (conj - c0)


def velocity_series(X, gX, g_nodes, M: int):
    """The same discrete U(x) as a Taylor series in the collocation point x (oracle.taylor).

    With x = tan(phi/2) and s_j = tan(psi_j/2) the kernel is rational in x,
    cot((phi - psi_j)/2) = (1 + x s_j) / (x - s_j), so
      U(x) = x [ (1/M) sum_j (g_j - g(x)) (1 + x s_j) / (x - s_j) - c0 ]
    is the function velocity() evaluates, here differentiated exactly in x: X is the series of
    the coordinate, gX the series of g at the points, g_nodes the node values (independent of x)."""
    from .taylor import Taylor
    _, s = nodes(M)
    Xb = Taylor({m: c[:, None] + 0.0 * s[None, :] for m, c in X.c.items()}, X.d, X.K)    # (n, M)
    gb = Taylor({m: c[:, None] + 0.0 * s[None, :] for m, c in gX.c.items()}, gX.d, gX.K)
    terms = (gb * (-1.0) + g_nodes[None, :]) * (Xb * s[None, :] + 1.0) / (Xb - s[None, :])
    conj = Taylor({m: c.sum(axis=1) / M for m, c in terms.c.items()}, terms.d, terms.K)
    c0 = (g_nodes * s).sum() / M
    return X * (conj - c0)


def hilbert_decaying(x, f, M: int):
    """H f(x) for a decaying f (no s*g factorisation): C[F](phi) - c0_f with the same rule.
    Used only by the tests that pin the quadrature to known transform pairs."""
    psi, s = nodes(M)
    phi = 2.0 * np.arctan(np.asarray(x, dtype=np.float64))
    fx = f(np.asarray(x, dtype=np.float64))
    fn = f(s)
    cot = 1.0 / np.tan(0.5 * (phi[:, None] - psi[None, :]))
    conj = ((fn[None, :] - fx[:, None]) * cot).sum(axis=1) / M
    c0 = (fn * s).sum() / M
    return conj - c0
