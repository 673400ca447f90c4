"""Pins for the oracle's residual operators against the PDEs themselves.

For each equation the time-dependent PDE is written out symbolically in the
physical variables (x, t), the self-similar ansatz phi_A = tau^{k_A} Phi_A(y),
y = x / tau^{1+lambda}, tau = 1 - t (paper, Methods, Eq. self-similar) is
substituted for concrete analytic test profiles Phi_A, and the result divided
by tau^{f_k} must equal the oracle's residual operator evaluated on the exact
derivatives of Phi_A.  A wrong exponent k_A, sign or transport term fails.

The Boussinesq lambda-inference rule printed in the paper (Methods,
"Identifying Admissible lambda Values", item 2) is then recovered from the
oracle's R_Theta: d^2/dy1^2 R_Theta at the origin vanishes iff
lambda = a + b dU1/dy1(0,0), with a, b read from tests/golden.
"""
import json
import os

import numpy as np
import pytest
import sympy as sp

from oracle import problems as Pb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")

x1, x2, t, Y1, Y2, lam = sp.symbols("x1 x2 t Y1 Y2 lam", real=True)
tau = 1 - t


def _phys(Phi, k, d):
    """tau^k Phi(x / tau^(1+lambda)) as an expression in x, t."""
    sub = {Y1: x1 / tau ** (1 + lam)}
    if d == 2:
        sub[Y2] = x2 / tau ** (1 + lam)
    return tau ** k * Phi.subs(sub)


def _num(expr, vals):
    return complex(sp.N(expr.subs(vals), 30)).real


def _check(pde_exprs, f_exps, oracle_R, yv, tv, lv):
    y1v, y2v = yv
    vals = {x1: y1v * (1 - tv) ** (1 + lv), x2: y2v * (1 - tv) ** (1 + lv), t: tv, lam: lv}
    for E, f, R in zip(pde_exprs, f_exps, oracle_R):
        lhs = _num(E, vals) / (1 - tv) ** f.subs(lam, lv)
        rhs = float(sp.N(R.subs({Y1: y1v, Y2: y2v, lam: lv}), 30))
        assert abs(lhs - rhs) <= 1e-10 * (1 + abs(rhs)), (lhs, rhs)


PTS = [((0.7, 0.3), 0.4, 0.8), ((-1.3, 0.9), 0.75, 1.9), ((0.2, 1.7), 0.1, 0.45)]


def test_burgers_reduction():
    U = sp.Rational(3, 10) * Y1 + sp.sin(Y1) / (2 + Y1**2)
    u = _phys(U, lam, 1)
    E = sp.diff(u, t) + u * sp.diff(u, x1)
    R = Pb.residual_burgers(lam, Y1, U, sp.diff(U, Y1))
    for (y, _), tv, lv in PTS:
        _check([E], [lam - 1], R, (y, 0.0), tv, lv)


def test_ccf_reduction():
    # U = H Theta scales like Theta because H commutes with dilations; the
    # transport structure is tested with an independent velocity profile.
    Th = Y1**2 / (1 + Y1**2) + sp.Rational(1, 5) * sp.cos(Y1)
    Uv = sp.atan(Y1) - sp.Rational(1, 3) * Y1 / (1 + Y1**4)
    th, u = _phys(Th, lam, 1), _phys(Uv, lam, 1)
    E = sp.diff(th, t) + u * sp.diff(th, x1)
    R = Pb.residual_ccf(lam, Y1, Th, sp.diff(Th, Y1), Uv)
    for (y, _), tv, lv in PTS:
        _check([E], [lam - 1], R, (y, 0.0), tv, lv)


def test_ipm_reduction():
    P = sp.cos(Y1) * sp.exp(-Y2 / 3) + Y2**2 / 5
    Psi = Y1 * (1 + Y2) / (2 + Y1**2 + Y2**2)
    rho, psi = _phys(P, lam, 2), _phys(Psi, 1 + 2 * lam, 2)
    u1, u2 = sp.diff(psi, x2), -sp.diff(psi, x1)
    E1 = sp.diff(rho, t) + u1 * sp.diff(rho, x1) + u2 * sp.diff(rho, x2)
    E2 = sp.diff(psi, x1, 2) + sp.diff(psi, x2, 2) - sp.diff(rho, x1)
    R = Pb.residual_ipm(lam, Y1, Y2, P, sp.diff(P, Y1), sp.diff(P, Y2), sp.diff(Psi, Y1),
                        sp.diff(Psi, Y2), sp.diff(Psi, Y1, 2), sp.diff(Psi, Y2, 2))
    for y, tv, lv in PTS:
        _check([E1, E2], [lam - 1, sp.Integer(-1)], R, y, tv, lv)


def test_ipm_stream_function_equation_from_darcy():
    """Delta psi = d1 rho follows from Darcy u = -grad p - (0, rho), div u = 0 and
    u = (d2 psi, -d1 psi): curl u = -d1 rho and curl u = -Delta psi."""
    X, Y = sp.symbols("X Y")
    p = sp.Function("p")(X, Y)
    rho = sp.Function("rho")(X, Y)
    u1 = -sp.diff(p, X)
    u2 = -sp.diff(p, Y) - rho
    curl = sp.diff(u2, X) - sp.diff(u1, Y)
    assert sp.simplify(curl + sp.diff(rho, X)) == 0
    psi = sp.Function("psi")(X, Y)
    curl_psi = sp.diff(-sp.diff(psi, X), X) - sp.diff(sp.diff(psi, Y), Y)
    assert sp.simplify(curl_psi + sp.diff(psi, X, 2) + sp.diff(psi, Y, 2)) == 0


def test_boussinesq_reduction():
    Om = Y1 * sp.exp(-(Y1**2 + Y2**2) / 4)
    Th = 1 / (1 + Y1**2) + Y2 / 7
    Psi = Y1 * Y2 * sp.cos(Y2 / 2) / (1 + Y1**2)
    om, th, psi = _phys(Om, -1, 2), _phys(Th, lam - 1, 2), _phys(Psi, 1 + 2 * lam, 2)
    u1, u2 = sp.diff(psi, x2), -sp.diff(psi, x1)
    E1 = sp.diff(om, t) + u1 * sp.diff(om, x1) + u2 * sp.diff(om, x2) - sp.diff(th, x1)
    E2 = sp.diff(th, t) + u1 * sp.diff(th, x1) + u2 * sp.diff(th, x2)
    E3 = sp.diff(psi, x1, 2) + sp.diff(psi, x2, 2) + om
    R = Pb.residual_boussinesq(lam, Y1, Y2, Om, sp.diff(Om, Y1), sp.diff(Om, Y2), Th,
                               sp.diff(Th, Y1), sp.diff(Th, Y2), sp.diff(Psi, Y1),
                               sp.diff(Psi, Y2), sp.diff(Psi, Y1, 2), sp.diff(Psi, Y2, 2))
    for y, tv, lv in PTS:
        _check([E1, E2, E3], [sp.Integer(-2), lam - 2, sp.Integer(-1)], R, y, tv, lv)


def _taylor_fields():
    """Generic polynomial profiles near the origin with the symmetry and wall
    conditions of the Boussinesq/IPM setting: Omega odd in y1, Theta/P even in y1,
    Psi odd in y1 and zero on the wall y2 = 0."""
    c = sp.symbols("o0:4 t0:6 p0:4", real=True)
    o, th, p = c[0:4], c[4:10], c[10:14]
    Om = Y1 * (o[0] + o[1] * Y2 + o[2] * Y1**2 + o[3] * Y2**2)
    Th = th[0] + th[1] * Y2 + th[2] * Y1**2 + th[3] * Y2**2 + th[4] * Y1**2 * Y2 + th[5] * Y1**4
    Psi = Y1 * Y2 * (p[0] + p[1] * Y2 + p[2] * Y1**2 + p[3] * Y2**2)
    return Om, Th, Psi, o, th, p


def test_boussinesq_lambda_inference_rule_from_paper():
    with open(GOLDEN) as f:
        g = json.load(f)["boussinesq_lambda_inference"]
    Om, Th, Psi, o, th, p = _taylor_fields()
    R = Pb.residual_boussinesq(lam, Y1, Y2, Om, sp.diff(Om, Y1), sp.diff(Om, Y2), Th,
                               sp.diff(Th, Y1), sp.diff(Th, Y2), sp.diff(Psi, Y1),
                               sp.diff(Psi, Y2), sp.diff(Psi, Y1, 2), sp.diff(Psi, Y2, 2))
    RTh = R[1]
    d11 = sp.expand(sp.diff(RTh, Y1, 2).subs({Y1: 0, Y2: 0}))
    dU1 = sp.diff(sp.diff(Psi, Y2), Y1).subs({Y1: 0, Y2: 0})  # U1 = d2 Psi
    sol = sp.solve(sp.Eq(d11, 0), lam)
    assert len(sol) == 1
    assert sp.simplify(sol[0] - (g["a"] + g["b"] * dU1)) == 0
    # the first-order condition is automatic: R_Theta is even in y1
    assert sp.simplify(sp.diff(RTh, Y1).subs({Y1: 0, Y2: 0})) == 0


def test_ipm_and_ccf_lambda_inference_consistency():
    """Same construction for IPM (derived, not printed): lambda = -2 - 2 dU1/dy1(0)."""
    _, Th, Psi, _, _, _ = _taylor_fields()
    R = Pb.residual_ipm(lam, Y1, Y2, Th, sp.diff(Th, Y1), sp.diff(Th, Y2), sp.diff(Psi, Y1),
                        sp.diff(Psi, Y2), sp.diff(Psi, Y1, 2), sp.diff(Psi, Y2, 2))
    d11 = sp.expand(sp.diff(R[0], Y1, 2).subs({Y1: 0, Y2: 0}))
    dU1 = sp.diff(sp.diff(Psi, Y2), Y1).subs({Y1: 0, Y2: 0})
    sol = sp.solve(sp.Eq(d11, 0), lam)
    assert sp.simplify(sol[0] - (-2 - 2 * dU1)) == 0
