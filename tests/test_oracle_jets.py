"""Pins for the oracle's jet arithmetic and complex-step derivatives.

The jets must agree with derivatives obtained a different way: complex-step in
y (first derivatives, exact to rounding), central differences of the
complex-step first derivatives (second derivatives), and closed forms.
"""
import numpy as np
import pytest

from oracle.jets import Jet
from oracle import problems as Pb
from paper_2509_14185_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_closed_forms_2d():
    rng = np.random.default_rng(0)
    y1, y2 = rng.uniform(-2, 2, 50), rng.uniform(-2, 2, 50)
    a, b = Jet.variable(y1, 0, 2), Jet.variable(y2, 1, 2)
    f = (a * a * b + (a * b).tanh()) / (1.0 + a * a + b * b).sqrt()
    # sympy-free closed forms for f = x^2 y + tanh(xy) over sqrt(1+x^2+y^2)
    import sympy as sp
    X, Y = sp.symbols("x y")
    F = (X**2 * Y + sp.tanh(X * Y)) / sp.sqrt(1 + X**2 + Y**2)
    fns = {k: sp.lambdify((X, Y), e, "numpy") for k, e in {
        "v": F, "1": sp.diff(F, X), "2": sp.diff(F, Y), "11": sp.diff(F, X, 2),
        "12": sp.diff(F, X, Y), "22": sp.diff(F, Y, 2)}.items()}
    np.testing.assert_allclose(f.v, fns["v"](y1, y2), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(f.g[0], fns["1"](y1, y2), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(f.g[1], fns["2"](y1, y2), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(f.h[0][0], fns["11"](y1, y2), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(f.h[0][1], fns["12"](y1, y2), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(f.h[1][0], fns["12"](y1, y2), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(f.h[1][1], fns["22"](y1, y2), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("eq,widths", [(Pb.BURGERS, [1, 6, 6, 1]), (Pb.CCF, [1, 6, 6, 1]),
                                       (Pb.IPM, [2, 6, 6, 2]), (Pb.BOUSSINESQ, [2, 6, 6, 3])])
def test_field_jets_vs_complex_step_in_y(eq, widths):
    """The ansatz fields' y-derivatives from jets equal complex-step derivatives of the
    field values in y (first order) and central differences of those (second order)."""
    w = I.small_case(eq, widths, 9, n_bnd=0, m=16)
    p = Pb.Problem(eq, widths, w.y, hilbert_m=16)
    d = p.d
    ys = w.y[:, :9]
    F = p.fields(w.theta, w.lam, ys)
    h = 1e-30

    def vals(yc):
        return [f.v for f in p.fields(w.theta, w.lam, yc)]

    for i in range(d):
        yc = ys.astype(np.complex128)
        yc[i] += 1j * h
        dv = [v.imag / h for v in vals(yc)]
        for a, f in enumerate(F):
            np.testing.assert_allclose(f.g[i], dv[a], rtol=1e-12, atol=1e-14 * np.max(np.abs(dv[a])))
        # second derivatives: central difference (in y_j) of the complex-step d/dy_i
        for j in range(d):
            e = 1e-5 * np.maximum(1.0, np.abs(ys[j]))
            yp = yc.copy(); yp[j] += e
            ym = yc.copy(); ym[j] -= e
            d2 = [(a_.imag - b_.imag) / h / (2 * e) for a_, b_ in zip(vals(yp), vals(ym))]
            for a, f in enumerate(F):
                scale = np.max(np.abs(f.h[i][j])) + np.max(np.abs(f.g[i]))
                np.testing.assert_allclose(f.h[i][j], d2[a], rtol=1e-6, atol=1e-7 * scale)


def test_complex_step_matches_central_differences():
    """J~ by complex step agrees with central differences (a pin of the oracle's
    Jacobian definition that does not reuse complex arithmetic)."""
    from oracle import gn
    for eq, widths in [(Pb.CCF, [1, 5, 5, 1]), (Pb.BOUSSINESQ, [2, 5, 5, 3])]:
        w = I.small_case(eq, widths, 10, n_bnd=3, m=16)
        p = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=w.y_norm, hilbert_m=16)
        cols = [0, 3, p.P // 2, p.P - 1, p.P]
        J = gn.jacobian(p, w.theta, w.lam, cols)
        x = np.concatenate([w.theta, [w.lam]])
        for c, j in enumerate(cols):
            e = 1e-6 * max(1.0, abs(x[j]))
            xp, xm = x.copy(), x.copy()
            xp[j] += e
            xm[j] -= e
            fd = (p.rows(xp[:-1], xp[-1]) - p.rows(xm[:-1], xm[-1])) / (2 * e)
            np.testing.assert_allclose(J[:, c], fd, rtol=1e-5, atol=1e-7 * np.max(np.abs(fd)))
