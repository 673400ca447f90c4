"""Damped Gauss-Newton step, written out from its definition (FP64).

Paper, Methods, "Second-order Optimizer": the loss is h = sum_i c_i |f_i|^2
and the step is theta <- theta - (G + gamma I)^{-1} grad h with G the
Gauss-Newton matrix and gamma a damping coefficient adapted by
Levenberg-Marquardt.  With the weighted rows r~ of problems.Problem.rows,
h = 1/2 |r~|^2, grad h = J~^T r~ and G = J~^T J~ exactly; lambda is the last
unknown (gradient training of lambda, "Identifying admissible lambda values",
item 1), so J~ has P + 1 columns.

Readings where the paper gives no constants (listed in the design notes):
Armijo backtracking with c1 = 1e-4, alpha = 1, 1/2, ... (at most 8 trials);
LM ratio rho = (h0 - h(alpha)) / (h0 - m(alpha)) with the undamped model
m(alpha) = h0 - alpha g.delta + alpha^2/2 delta.G.delta; gamma *= 1.5 if
rho < 1/4, gamma *= 2/3 if rho > 3/4; no accepted trial -> theta unchanged,
gamma *= 10; Cholesky failure -> gamma *= 10, at most 5 retries.
"""
from __future__ import annotations

import numpy as np

STEP_OK = 0
WARN_NO_DECREASE = 1
ERR_NOT_SPD = -5

ARMIJO_C1 = 1e-4
MAX_TRIALS = 8
MAX_CHOL_RETRIES = 5
CS_STEP = 1e-30


def jacobian(problem, theta, lam, cols=None):
    """J~[:, j] = d r~ / d(theta, lambda)_j by complex-step differentiation
    (Squire & Trapp 1998): Im r~(x + i h e_j) / h, exact to rounding for
    analytic r~.  `cols` selects columns (index P is lambda)."""
    P = problem.P
    cols = range(P + 1) if cols is None else cols
    out = []
    th = theta.astype(np.complex128)
    for j in cols:
        if j == P:
            r = problem.rows(th, lam + 1j * CS_STEP)
        else:
            tj = th.copy()
            tj[j] += 1j * CS_STEP
            r = problem.rows(tj, complex(lam))
        out.append(r.imag / CS_STEP)
    return np.stack(out, axis=1)


def cholesky(A):
    """Textbook column Cholesky A = L L^T; returns (L, ok).  ok is False as soon
    as a pivot is not positive (the matrix is not numerically SPD)."""
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        s = A[j, j] - np.dot(L[j, :j], L[j, :j])
        if not (s > 0.0) or not np.isfinite(s):
            return L, False
        L[j, j] = np.sqrt(s)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L, True


def cholesky_solve(L, b):
    """Solve L L^T x = b by forward then backward substitution."""
    n = L.shape[0]
    z = np.zeros_like(b)
    for i in range(n):
        z[i] = (b[i] - np.dot(L[i, :i], z[:i])) / L[i, i]
    x = np.zeros_like(b)
    for i in range(n - 1, -1, -1):
        x[i] = (z[i] - np.dot(L[i + 1:, i], x[i + 1:])) / L[i, i]
    return x


def damped_solve(G, g, gamma):
    """delta = (G + gamma I)^{-1} g with gamma escalation on factorisation failure."""
    n = G.shape[0]
    retries = 0
    while True:
        L, ok = cholesky(G + gamma * np.eye(n))
        if ok:
            return cholesky_solve(L, g), gamma, retries, True
        if retries == MAX_CHOL_RETRIES:
            return None, gamma, retries, False
        gamma *= 10.0
        retries += 1


def gn_step_generic(rows_fn, jac_fn, x, gamma):
    """One damped GN step on the unknowns x (theta with lambda appended).

    rows_fn(x) -> r~, jac_fn(x) -> J~.  Returns (x_new, gamma_new, info)."""
    r = rows_fn(x)
    J = jac_fn(x)
    h0 = 0.5 * float(r @ r)
    g = J.T @ r
    G = J.T @ J
    info = {"loss_before": h0, "chol_retries": 0, "alpha": 0.0, "rho": 0.0,
            "loss_after": h0, "status": STEP_OK, "gamma_used": gamma}
    delta, gamma, retries, ok = damped_solve(G, g, gamma)
    info["chol_retries"] = retries
    info["gamma_used"] = gamma
    if not ok:
        info["status"] = ERR_NOT_SPD
        return x, gamma, info
    gd = float(g @ delta)
    Jd = J @ delta
    dGd = float(Jd @ Jd)
    alpha = 1.0
    for _ in range(MAX_TRIALS):
        xt = x - alpha * delta
        rt = rows_fn(xt)
        ht = 0.5 * float(rt @ rt) if np.all(np.isfinite(rt)) else np.inf
        if ht <= h0 - ARMIJO_C1 * alpha * gd:
            pred = alpha * gd - 0.5 * alpha * alpha * dGd
            rho = (h0 - ht) / pred if pred != 0.0 else 1.0
            if rho < 0.25:
                gamma *= 1.5
            elif rho > 0.75:
                gamma *= 2.0 / 3.0
            info.update(alpha=alpha, rho=rho, loss_after=ht, delta=delta, g=g, G=G)
            return xt, gamma, info
        alpha *= 0.5
    info.update(status=WARN_NO_DECREASE, delta=delta, g=g, G=G)
    return x, gamma * 10.0, info


def gn_step(problem, theta, lam, gamma):
    """One damped GN step of a profile fit: returns (theta, lambda, gamma, info)."""
    P = problem.P

    def rows_fn(x):
        return problem.rows(x[:P], x[P])

    def jac_fn(x):
        return jacobian(problem, x[:P], x[P])

    x = np.concatenate([theta, [lam]])
    xn, gamma, info = gn_step_generic(rows_fn, jac_fn, x, gamma)
    return xn[:P].copy(), float(xn[P]), gamma, info
