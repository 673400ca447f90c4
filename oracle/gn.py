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


# ---------------------------------------------------------------------------
# The paper's own curvature estimate (Methods, "Second-order Optimizer"): an
# exponential moving average over iterations of an unbiased rank-1 estimate of
# G from one product with the Jacobian, and per-iteration learning rate and
# momentum chosen in closed form by the quadratic-model rule of Martens &
# Grosse (2015).  Readings (the paper gives no constants and defers to
# kfac-jax): the sign vector v (independent +-1 entries, so E[v v^T] = I and
# E[u u^T] = G for u = J~^T v) is an input; the average starts at the first
# sample; the direction is Delta = -(G_ema + gamma I)^{-1} g; (alpha, mu)
# minimise the damped model M(d) = g.d + 1/2 d.(G + gamma I).d over
# d = alpha Delta + mu v_prev with the exact G applied through J~ products
# (mu = 0 while v_prev = 0); the update is applied whenever the new loss is
# finite; gamma follows the same Levenberg-Marquardt rule as the exact step,
# with rho measured against the undamped model.
# ---------------------------------------------------------------------------
def rank1_estimate(J, v):
    """u = J^T v; u u^T estimates J^T J without bias for independent +-1 signs v."""
    return J.T @ v


def mg_coefficients(C_dd, C_dv, C_vv, g_d, g_v, have_v):
    """(alpha, mu) minimising g.d + 1/2 d.C.d over d = alpha Delta + mu v:
    the 2 x 2 normal equations [C_dd C_dv; C_dv C_vv] [alpha; mu] = -[g_d; g_v]
    (mu = 0 without a previous update, or when the 2 x 2 system is singular)."""
    if have_v:
        det = C_dd * C_vv - C_dv * C_dv
        if det > 0.0 and np.isfinite(det):
            alpha = (-g_d * C_vv + g_v * C_dv) / det
            mu = (-g_v * C_dd + g_d * C_dv) / det
            return alpha, mu
    return -g_d / C_dd, 0.0


def ema_step_generic(rows_fn, jac_fn, x, gamma, G_ema, v_prev, signs, beta, first):
    """One step of the EMA rank-1 optimiser on the unknowns x (theta with lambda appended).
    Returns (x_new, gamma_new, G_ema_new, v_new, info)."""
    r = rows_fn(x)
    J = jac_fn(x)
    h0 = 0.5 * float(r @ r)
    g = J.T @ r
    u = rank1_estimate(J, signs)
    G_new = np.outer(u, u) if first else beta * G_ema + (1.0 - beta) * np.outer(u, u)
    info = {"loss_before": h0, "loss_after": h0, "alpha": 0.0, "mu": 0.0, "rho": 0.0,
            "chol_retries": 0, "status": STEP_OK, "gamma_used": gamma}
    delta, gamma, retries, ok = damped_solve(G_new, g, gamma)
    info["chol_retries"] = retries
    info["gamma_used"] = gamma
    if not ok:
        info["status"] = ERR_NOT_SPD
        return x, gamma, G_new, v_prev, info
    D = -delta                                   # the direction Delta
    JD, Jv = J @ D, J @ v_prev
    C_dd = float(JD @ JD) + gamma * float(D @ D)
    C_dv = float(JD @ Jv) + gamma * float(D @ v_prev)
    C_vv = float(Jv @ Jv) + gamma * float(v_prev @ v_prev)
    g_d, g_v = float(g @ D), float(g @ v_prev)
    have_v = (not first) and float(v_prev @ v_prev) > 0.0
    alpha, mu = mg_coefficients(C_dd, C_dv, C_vv, g_d, g_v, have_v)
    d = alpha * D + mu * v_prev
    xt = x + d
    rt = rows_fn(xt)
    ht = 0.5 * float(rt @ rt) if np.all(np.isfinite(rt)) else np.inf
    Jd = alpha * JD + mu * Jv
    model = alpha * g_d + mu * g_v + 0.5 * float(Jd @ Jd)      # undamped model change M(d) - M(0)
    info.update(alpha=alpha, mu=mu, delta=delta, g=g, G_ema=G_new)
    if not np.isfinite(ht):
        info["status"] = WARN_NO_DECREASE
        return x, gamma * 10.0, G_new, np.zeros_like(v_prev), info
    rho = (ht - h0) / model if model != 0.0 else 1.0
    if rho < 0.25:
        gamma *= 1.5
    elif rho > 0.75:
        gamma *= 2.0 / 3.0
    info.update(rho=rho, loss_after=ht)
    return xt, gamma, G_new, d, info


def ema_step(problem, theta, lam, gamma, G_ema, v_prev, signs, beta, first):
    """EMA rank-1 step of a profile fit: returns (theta, lambda, gamma, G_ema, v_prev, info)."""
    P = problem.P

    def rows_fn(x):
        return problem.rows(x[:P], x[P])

    def jac_fn(x):
        return jacobian(problem, x[:P], x[P])

    x = np.concatenate([theta, [lam]])
    xn, gamma, G_new, v_new, info = ema_step_generic(rows_fn, jac_fn, x, gamma, G_ema, v_prev, signs, beta,
                                                     first)
    return xn[:P].copy(), float(xn[P]), gamma, G_new, v_new, info
