"""Pins for the truncated Taylor arithmetic of oracle/taylor.py (the derivative losses' y-jets):
every partial derivative up to order 4 of composite expressions (products, quotients, powers,
exp, tanh, cos, sin) against sympy's symbolic derivatives at several points, in 1 and 2
variables; d/dy_i of a series against the series of the derivative."""
from math import factorial

import numpy as np
import pytest
import sympy as sp

from oracle.taylor import Taylor, multi_indices


def check(expr_fn, sym_expr, syms, pts, K=4, rtol=1e-11):
    d = len(syms)
    ys = [np.array(p, dtype=np.float64) for p in pts]
    T = expr_fn(*[Taylor.variable(ys[i], i, d, K) for i in range(d)])
    for a in multi_indices(d, K):
        e = sym_expr
        for i, k in enumerate(a):
            if k:
                e = sp.diff(e, syms[i], k)
        f = sp.lambdify(syms, e, "numpy")
        want = np.broadcast_to(np.asarray(f(*ys), dtype=np.float64), ys[0].shape)
        got = T.deriv(a)
        assert np.allclose(got, want, rtol=rtol, atol=rtol * (1 + np.max(np.abs(want)))), (a, got, want)


def test_one_variable_composites():
    y = sp.Symbol("y")
    pts = [[-1.3, 0.2, 0.7, 2.5]]
    check(lambda t: (t * t + 1.0).pow(-0.37) * t.tanh(), (y ** 2 + 1) ** sp.Rational(-37, 100) * sp.tanh(y), [y], pts)
    check(lambda t: (t.sin() * 2.0 + t.cos()).exp() / (3.0 + t * t), sp.exp(2 * sp.sin(y) + sp.cos(y)) / (3 + y ** 2),
          [y], pts)
    check(lambda t: (1.0 + t * t).sqrt() - t, sp.sqrt(1 + y ** 2) - y, [y], pts)


def test_two_variable_composites():
    y1, y2 = sp.symbols("y1 y2")
    pts = [[0.3, -1.1, 2.0], [0.8, 0.4, -0.6]]
    check(lambda a, b: (a * b + b.tanh()).exp() * (1.0 + a * a + b * b).pow(-0.8),
          sp.exp(y1 * y2 + sp.tanh(y2)) * (1 + y1 ** 2 + y2 ** 2) ** sp.Rational(-4, 5), [y1, y2], pts)
    check(lambda a, b: b / (1.0 + a * a + b * b).sqrt() * (a * 3.0).sin(),
          y2 / sp.sqrt(1 + y1 ** 2 + y2 ** 2) * sp.sin(3 * y1), [y1, y2], pts)


def test_diff_is_the_series_of_the_derivative():
    y1, y2 = sp.symbols("y1 y2")
    pts = [np.array([0.3, -0.7]), np.array([1.2, 0.5])]
    a, b = Taylor.variable(pts[0], 0, 2, 4), Taylor.variable(pts[1], 1, 2, 4)
    f = (a * b).tanh() * (a + 2.0).pow(1.5)
    g = f.diff(1)
    assert g.K == 3
    e = sp.diff(sp.tanh(y1 * y2) * (y1 + 2) ** sp.Rational(3, 2), y2)
    for m in multi_indices(2, 3):
        em = e
        for i, k in enumerate(m):
            if k:
                em = sp.diff(em, [y1, y2][i], k)
        want = sp.lambdify([y1, y2], em, "numpy")(*pts)
        np.testing.assert_allclose(g.deriv(m), want, rtol=1e-11, atol=1e-12)


def test_coefficients_are_derivatives_over_factorials():
    t = Taylor.variable(np.array([0.4]), 0, 1, 4).exp()
    for n in range(5):
        assert t.c[(n,)][0] == pytest.approx(np.exp(0.4) / factorial(n), rel=1e-15)
