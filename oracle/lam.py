"""Strategies for the blow-up rate lambda (FP64), written out from the paper.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper, Methods, "Identifying Admissible lambda Values":
  item 2 (lambda inference): differentiate the self-similar equation, evaluate
    it at the origin and require it to vanish; this gives lambda explicitly in
    terms of field values there, used as a direct update rule.  The paper
    prints the Boussinesq rule lambda = -3 - 2 d1 U1(0, 0).  The same steps on
    this project's residual operators give (derived in the design notes and
    pinned symbolically by the PDE-reduction tests)
        IPM         lambda = -2 - 2 d1 U1(0, 0)
        CCF         lambda = -2 - 2 U'(0)
        Boussinesq  lambda = -3 - 2 d1 U1(0, 0)
    with U1 = d2 Psi in 2D (so d1 U1 = d12 Psi) and U = x H[Theta/x] in CCF,
    U'(0) = H[g](0).  Burgers has U'(0) = -1 for every lambda: no rule.
  item 3 (funnel inference): train with lambda held fixed, take r_hat(lambda)
    = the residual of largest absolute value (with its sign) in a small
    neighbourhood of the origin, and move lambda by the secant method on the
    last two (lambda, r_hat) pairs; the first move is lambda_1 = lambda_0 +
    dlambda.  Reading: the printed update puts lambda_n in front of the
    correction computed from the pair anchored at lambda_{n-1}; the text calls
    it the secant formula, so the secant zero through the last two pairs is
    used:  lambda_{n+1} = lambda_n - r_n (lambda_n - lambda_{n-1}) / (r_n - r_{n-1}).
  Training "with this fixed lambda value": a damped GN step on theta alone.
"""
from __future__ import annotations

import numpy as np

from . import gn as ogn
from . import hilbert
from .problems import BOUSSINESQ, BURGERS, CCF, IPM


def frozen_gn_step(problem, theta, lam, gamma):
    """One damped GN step with lambda held fixed: the unknowns are theta only."""
    P = problem.P

    def rows_fn(x):
        return problem.rows(x, lam)

    def jac_fn(x):
        return ogn.jacobian(problem, x, lam, cols=range(P))

    th, gamma, info = ogn.gn_step_generic(rows_fn, jac_fn, np.asarray(theta, dtype=np.float64), gamma)
    return th.copy(), float(lam), gamma, info


def origin_field_jets(problem, theta, lam):
    """Field jets Phi_A (value, gradient, Hessian) at the origin y = 0."""
    ys = np.zeros((problem.d, 1))
    return problem.fields(theta, lam, ys)


def ccf_dU_at_origin(problem, theta, lam):
    """U'(0) = H[g](0) for U = x H[g], g = Theta / x, by the discrete operator of
    hilbert.py at x = 0 (where g(0) = 0): (1/M) sum_j g_j cot(-psi_j / 2) - c0."""
    psi, s = hilbert.nodes(problem.M)
    g_nodes = problem.fields(theta, lam, s.reshape(1, -1), extra_g=True)[1].v
    conj = np.sum(g_nodes / np.tan(-0.5 * psi)) / problem.M
    c0 = np.sum(g_nodes * s) / problem.M
    return float(conj - c0)


def lambda_inference(problem, theta, lam):
    """The lambda-inference rule of item 2 evaluated on the current network."""
    if problem.eq == BOUSSINESQ or problem.eq == IPM:
        psi = origin_field_jets(problem, theta, lam)[-1]
        d1U1 = float(psi.h[0][1][0])          # U1 = d2 Psi  ->  d1 U1 = d12 Psi
        base = -3.0 if problem.eq == BOUSSINESQ else -2.0
        return base - 2.0 * d1U1
    if problem.eq == CCF:
        return -2.0 - 2.0 * ccf_dU_at_origin(problem, theta, lam)
    raise ValueError("Burgers: U'(0) = -1 for every lambda, the rule carries no information")


def signed_max_residual(problem, theta, lam, radius):
    """r_hat of item 3: over the interior points with |y| <= radius and every equation,
    the unweighted residual of largest absolute value, with its sign (first point, then
    first equation, on ties).  Returns (r_hat, point index); (0.0, -1) if no point."""
    ys = problem.y
    near = np.nonzero(np.sqrt(np.sum(ys * ys, axis=0)) <= radius)[0]
    if near.size == 0:
        return 0.0, -1
    R = problem.interior_residuals(theta, lam)
    best, arg, best_i = -1.0, 0.0, -1
    for i in near:
        for k in range(problem.ne):
            v = float(R[k][i])
            if abs(v) > best:
                best, arg, best_i = abs(v), v, int(i)
    return arg, best_i


def funnel_next(lams, rhats, dlam):
    """Next lambda of funnel inference from the history (lambda_0..n, r_hat_0..n)."""
    n = len(lams)
    if n == 0 or n != len(rhats):
        raise ValueError("history of equal, non-zero length expected")
    if n == 1:
        return float(lams[0] + dlam)
    l0, l1 = lams[-2], lams[-1]
    r0, r1 = rhats[-2], rhats[-1]
    if r1 == r0:
        raise ZeroDivisionError("secant undefined: equal r_hat")
    return float(l1 - r1 * (l1 - l0) / (r1 - r0))
