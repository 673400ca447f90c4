"""Pins of the oracle's lambda strategies (oracle/lam.py) against things other than itself:
finite differences of the field values, the discrete Hilbert velocity near the origin,
brute force over the residuals, closed-form secant behaviour, and a central-difference
Jacobian for the frozen-lambda step."""
import warnings

import numpy as np
import pytest

from oracle import gn as ogn
from oracle import hilbert
from oracle import lam as olam
from oracle import problems as Pb
from paper_2509_14185_gb300 import inputs as I

warnings.filterwarnings("ignore", category=RuntimeWarning)


def problem(eq, widths, n, nb=0, seed=11, m=64):
    w = I.small_case(eq, widths, n, n_bnd=nb, seed=seed, m=m)
    p = Pb.Problem(w.equation, w.widths, w.y, w.y_bnd if w.y_bnd.size else None, w.rho,
                   y_norm=w.y_norm, c_norm=w.c_norm, hilbert_m=w.hilbert_m)
    return w, p


@pytest.mark.parametrize("eq", [I.IPM, I.BOUSSINESQ])
def test_lambda_inference_2d_matches_finite_differences(eq):
    nf = 2 if eq == I.IPM else 3
    w, p = problem(eq, [2, 12, 12, nf], 20, nb=4)
    th = w.theta + 0.3 * np.sin(np.arange(p.P))      # a non-trivial network
    lam = w.lam
    h = 1e-4
    pts = np.array([[h, h, -h, -h], [h, -h, h, -h]])
    psi = p.fields(th, lam, pts)[-1].v
    d12 = (psi[0] - psi[1] - psi[2] + psi[3]) / (4 * h * h)   # central mixed difference
    base = -3.0 if eq == I.BOUSSINESQ else -2.0
    got = olam.lambda_inference(p, th, lam)
    assert got == pytest.approx(base - 2.0 * d12, rel=1e-6, abs=1e-8)


def test_lambda_inference_ccf_matches_velocity_near_origin():
    """U'(0) = lim U(x)/x: the discrete velocity at small x over x converges (O(x^2))."""
    w, p = problem(I.CCF, [1, 10, 10, 1], 30, m=64)
    th = w.theta + 0.2 * np.cos(np.arange(p.P))
    lam = w.lam
    _, s = hilbert.nodes(p.M)
    g_nodes = p.fields(th, lam, s.reshape(1, -1), extra_g=True)[1].v
    vals = []
    for x in (1e-3, 5e-4):
        gx = p.fields(th, lam, np.array([[x]]), extra_g=True)[1].v
        vals.append(hilbert.velocity(np.array([x]), gx, g_nodes, p.M)[0] / x)
    dU0 = olam.ccf_dU_at_origin(p, th, lam)
    assert abs(vals[1] - dU0) < 0.3 * abs(vals[0] - dU0) + 1e-12     # converging to it
    assert dU0 == pytest.approx(vals[1], rel=1e-5, abs=1e-9)
    assert olam.lambda_inference(p, th, lam) == pytest.approx(-2.0 - 2.0 * dU0, rel=1e-15)


def test_lambda_inference_burgers_has_no_rule():
    w, p = problem(I.BURGERS, [1, 6, 1], 10)
    with pytest.raises(ValueError):
        olam.lambda_inference(p, w.theta, w.lam)


def test_signed_max_residual_brute_force_and_edges():
    w, p = problem(I.IPM, [2, 8, 8, 2], 60, nb=5)
    th = w.theta
    R = p.interior_residuals(th, w.lam)
    r = np.sqrt(np.sum(p.y ** 2, axis=0))
    radius = np.median(r)
    cand = [(abs(R[k][i]), R[k][i], i) for i in range(p.n) for k in range(p.ne) if r[i] <= radius]
    best = max(cand, key=lambda c: c[0])
    val, idx = olam.signed_max_residual(p, th, w.lam, radius)
    assert val == best[1] and idx == best[2]
    assert olam.signed_max_residual(p, th, w.lam, 0.5 * r.min()) == (0.0, -1)
    # over every point: the global max |R|, and its sign follows the residual's
    val_all, i_all = olam.signed_max_residual(p, th, w.lam, np.inf)
    assert abs(val_all) == max(np.max(np.abs(Rk)) for Rk in R)
    assert any(val_all == R[k][i_all] for k in range(p.ne))


def test_funnel_secant_closed_forms():
    # first move: lambda_0 + dlambda
    assert olam.funnel_next([0.7], [0.3], 0.01) == pytest.approx(0.71)
    # linear r(lambda) = a (lambda - lambda*): one secant step lands on lambda* exactly
    a, ls = -3.7, 0.6057
    r = lambda x: a * (x - ls)
    lams = [0.5, 0.52]
    nxt = olam.funnel_next(lams, [r(x) for x in lams], 0.02)
    assert nxt == pytest.approx(ls, rel=1e-14)
    # the formula as printed (lambda_n in front of the lambda_{n-1}-anchored correction) does not
    lit = lams[1] - r(lams[0]) * (lams[0] - lams[1]) / (r(lams[0]) - r(lams[1]))
    assert abs(lit - ls) > 1e-3
    # a smooth nonlinear r converges superlinearly to its root
    f = lambda x: np.tanh(4.0 * (x - 0.4703)) + 0.3 * (x - 0.4703) ** 2
    hist = [0.40]
    rh = [f(0.40)]
    for _ in range(8):
        hist.append(olam.funnel_next(hist, rh, 0.01))
        rh.append(f(hist[-1]))
        if abs(rh[-1]) < 1e-15:
            break
    assert abs(hist[-1] - 0.4703) < 1e-12
    with pytest.raises(ZeroDivisionError):
        olam.funnel_next([0.1, 0.2], [1.0, 1.0], 0.1)


def test_frozen_step_matches_central_difference_jacobian():
    """The frozen-lambda step keeps lambda and equals the same damped step built from a
    central-difference Jacobian in theta (an independent derivative route)."""
    w, p = problem(I.BURGERS, [1, 6, 6, 1], 40)
    th0 = w.theta
    lam = w.lam
    th1, lam1, gam1, info = olam.frozen_gn_step(p, th0, lam, 1e-3)
    assert lam1 == lam and info["status"] == 0

    def jac_fd(x):
        cols = []
        for j in range(p.P):
            e = np.zeros(p.P)
            e[j] = 1e-6 * max(1.0, abs(x[j]))
            cols.append((p.rows(x + e, lam) - p.rows(x - e, lam)) / (2 * e[j]))
        return np.stack(cols, axis=1)

    th_fd, gam_fd, info_fd = ogn.gn_step_generic(lambda x: p.rows(x, lam), jac_fd, th0.copy(), 1e-3)
    assert info_fd["alpha"] == info["alpha"]
    assert np.max(np.abs(th_fd - th1)) <= 1e-5 * np.max(np.abs(th1 - th0))
