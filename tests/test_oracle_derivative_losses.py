"""Pins for the oracle's derivative losses (Methods, "Training Loss": the d1 and d2 losses
differentiate the residuals in y; rows sqrt(2 c rho / (N N_E d^n)) d^n R).

* Closed forms: Burgers at lambda = 1/2 (U^3 + U + y = 0) and lambda = 1/4 (U^5 + U + y = 0)
  solve R = 0 for every y, so every y-derivative of R vanishes.  U's Taylor series comes from
  implicit differentiation (sympy), not from the network or the jet code.
* The network path: d1 values equal the complex-step y-derivative of the d0 residual function
  (no Taylor code involved); d2 values equal central differences of those.
* The Taylor field series agree with the second-order Jet fields (two implementations).
* The loss gains exactly c_d1 / (N N_E d) sum rho (d R)^2 (with d R by complex step), and
  g = J~^T r~ stays the gradient of h (complex step of h in theta through the series).
* CCF: the discrete Hilbert velocity differentiated in the collocation point; its rational
  form has the circle-map form's value, and d1 / d2 match central differences of the d0 residual.
"""
from math import factorial

import numpy as np
import pytest
import sympy as sp

from oracle import gn
from oracle import hilbert
from oracle import problems as Pb
from oracle.taylor import Taylor
from paper_2509_14185_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def implicit_series(power, ys, K):
    """U(y) with U^power + U + y = 0 (the real root) as a Taylor series of order K at ys."""
    U_, y_ = sp.symbols("U y")
    F = U_ ** power + U_ + y_
    Uv = np.array([np.real([r for r in np.roots([1.0] + [0.0] * (power - 2) + [1.0, y0])
                            if abs(r.imag) < 1e-9][0]) for y0 in ys])
    c = {(0,): Uv}
    for n in range(1, K + 1):
        dn = sp.lambdify([U_, y_], sp.idiff(F, U_, y_, n), "numpy")
        c[(n,)] = np.asarray(dn(Uv, ys), dtype=np.float64) / factorial(n)
    return Taylor(c, 1, K)


@pytest.mark.parametrize("power,lam", [(3, 0.5), (5, 0.25)])
def test_burgers_closed_forms_have_flat_residuals(power, lam):
    ys = np.array([-3.0, -1.2, -0.4, 0.3, 0.9, 2.5])
    U = implicit_series(power, ys, 4)
    Y = Taylor.variable(ys, 0, 1, 4)
    (R,) = Pb.residual_burgers(lam, Y, U, U.diff(0))
    scale = np.max(np.abs(U.v)) + np.max(np.abs(ys))
    for n, S in enumerate([R, R.diff(0), R.diff(0).diff(0)]):
        assert np.max(np.abs(S.v)) <= 1e-13 * scale ** 2, n
    # and a slightly wrong lambda leaves them visibly non-zero
    (Rw,) = Pb.residual_burgers(lam + 1e-3, Y, U, U.diff(0))
    assert np.max(np.abs(Rw.diff(0).v)) > 1e-6


CASES = [(Pb.BURGERS, [1, 6, 6, 1]), (Pb.IPM, [2, 5, 5, 2]), (Pb.BOUSSINESQ, [2, 5, 5, 3])]


@pytest.mark.parametrize("eq,widths", CASES)
def test_d1_is_the_y_derivative_of_the_residual(eq, widths):
    w = I.small_case(eq, widths, 7, n_bnd=2, m=16, seed=2)
    p = Pb.Problem(eq, widths, w.y, w.y_bnd, hilbert_m=16, output_map=0)
    ys = w.y
    D1 = p.d1_residuals(w.theta, w.lam, ys)          # (ne, d, n)
    h = 1e-30
    for i in range(p.d):
        yc = ys.astype(np.complex128)
        yc[i] += 1j * h
        Rc = p.interior_residuals(w.theta, w.lam, yc)
        for k in range(p.ne):
            want = Rc[k].imag / h
            np.testing.assert_allclose(D1[k, i], want, rtol=1e-11, atol=1e-12 * np.max(np.abs(want)))


@pytest.mark.parametrize("eq,widths", CASES)
def test_d2_is_the_second_y_derivative(eq, widths):
    w = I.small_case(eq, widths, 5, n_bnd=2, m=16, seed=3)
    p = Pb.Problem(eq, widths, w.y, w.y_bnd, hilbert_m=16)
    ys = w.y
    D2 = p.d2_residuals(w.theta, w.lam, ys)          # (ne, d, d, n)
    e = 1e-5
    for j in range(p.d):
        out = []
        for s in (1.0, -1.0):
            yj = ys.copy()
            yj[j] += s * e
            out.append(p.d1_residuals(w.theta, w.lam, yj))
        fd = (out[0] - out[1]) / (2 * e)                # d/dy_j of d R / d y_i: (ne, d, n)
        for k in range(p.ne):
            for i in range(p.d):
                np.testing.assert_allclose(D2[k, i, j], fd[k, i], rtol=1e-6, atol=1e-7 * np.max(np.abs(fd[k, i])))
    # symmetric in (i, j)
    if p.d == 2:
        np.testing.assert_allclose(D2[:, 0, 1], D2[:, 1, 0], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("eq,widths", CASES + [(Pb.CCF, [1, 5, 1])])
def test_taylor_fields_match_the_jet_fields(eq, widths):
    w = I.small_case(eq, widths, 6, m=16, seed=4)
    p = Pb.Problem(eq, widths, w.y, hilbert_m=16)
    FJ = p.fields(w.theta, w.lam, w.y)
    FT = p.fields(w.theta, w.lam, w.y, order=2)
    for a, b in zip(FJ, FT):
        np.testing.assert_allclose(b.v, a.v, rtol=1e-13, atol=1e-300)
        for i in range(p.d):
            e_i = tuple(1 if k == i else 0 for k in range(p.d))
            np.testing.assert_allclose(b.deriv(e_i), a.g[i], rtol=1e-12, atol=1e-13 * np.max(np.abs(a.g[i])))
            for j in range(p.d):
                e_ij = tuple((1 if k == i else 0) + (1 if k == j else 0) for k in range(p.d))
                np.testing.assert_allclose(b.deriv(e_ij), a.h[i][j], rtol=1e-11,
                                           atol=1e-12 * np.max(np.abs(a.h[i][j])))


@pytest.mark.parametrize("eq,widths", CASES)
def test_loss_gains_the_d1_term_and_gradient(eq, widths):
    w = I.small_case(eq, widths, 6, n_bnd=2, m=16, seed=6)
    y1 = w.y[:, :4] * 1.3
    rho1 = np.array([0.5, 1.0, 2.0, 1.5])
    p0 = Pb.Problem(eq, widths, w.y, w.y_bnd, hilbert_m=16)
    p1 = Pb.Problem(eq, widths, w.y, w.y_bnd, hilbert_m=16, y_d1=y1, rho_d1=rho1, c_d1=0.7, y_d2=y1[:, :3], c_d2=0.2)
    assert p1.n_rows == p0.n_rows + 4 * p1.ne * p1.d + 3 * p1.ne * p1.d ** 2
    # d1 part of the loss from complex-step y-derivatives of the d0 residual (no Taylor code)
    h = 1e-30
    s1 = 0.0
    for i in range(p1.d):
        yc = y1.astype(np.complex128)
        yc[i] += 1j * h
        for Rk in p1.interior_residuals(w.theta, w.lam, yc):
            s1 += np.sum(rho1 * (Rk.imag / h) ** 2)
    D2 = p1.d2_residuals(w.theta, w.lam)
    want = p0.loss(w.theta, w.lam) + 0.7 * s1 / (4 * p1.ne * p1.d) + 0.2 * np.sum(D2 ** 2) / (3 * p1.ne * p1.d ** 2)
    assert p1.loss(w.theta, w.lam) == pytest.approx(want, rel=1e-11)
    # g = J~^T r~ is the gradient of h with the derivative rows (complex step of h in theta)
    J = gn.jacobian(p1, w.theta, w.lam)
    g = J.T @ p1.rows(w.theta, w.lam)
    x = np.concatenate([w.theta, [w.lam]]).astype(np.complex128)
    for j in [0, p1.P // 2, p1.P]:
        xc = x.copy()
        xc[j] += 1j * 1e-30
        r = p1.rows(xc[:-1], xc[-1])
        dh = (0.5 * np.sum(r * r)).imag / 1e-30
        assert abs(dh - g[j]) <= 1e-10 * (abs(g[j]) + 1e-3 * np.max(np.abs(g)))


def test_ccf_velocity_series_is_the_discrete_operator():
    """The rational form of the discrete Hilbert velocity (Taylor series in x) has the value
    of the circle-map form the d0 residual uses, at every point."""
    from oracle import hilbert
    w = I.small_case(Pb.CCF, [1, 6, 1], 9, m=32, seed=3)
    p = Pb.Problem(Pb.CCF, [1, 6, 1], w.y, hilbert_m=32)
    Th, g = p.fields(w.theta, w.lam, w.y, extra_g=True)
    _, s = hilbert.nodes(32)
    gn_ = p.fields(w.theta, w.lam, s.reshape(1, -1), extra_g=True)[1].v
    U0 = hilbert.velocity(w.y[0], g.v, gn_, 32)
    _, gT = p.fields(w.theta, w.lam, w.y, extra_g=True, order=2)
    UT = hilbert.velocity_series(Taylor.variable(w.y[0], 0, 1, 2), gT, gn_, 32)
    # the two forms round the near-singular kernel terms differently: bound the difference by
    # rounding of the sum of the terms' magnitudes, |x| (1/M) sum_j |g_j - g(x)| |cot|
    x = w.y[0]
    phi = 2.0 * np.arctan(x)
    psi, _ = hilbert.nodes(32)
    mag = np.abs(x) * (np.abs(gn_[None, :] - g.v[:, None]) / np.abs(np.tan(0.5 * (phi[:, None] - psi[None, :])))
                       ).sum(axis=1) / 32
    assert np.all(np.abs(UT.v - U0) <= 1e-14 * (mag + np.abs(U0)))


def test_ccf_d1_and_d2_are_y_derivatives_of_the_d0_residual():
    """CCF's d1 / d2 values against central differences of the d0 residual function (whose
    velocity casts x to real, so no complex step here)."""
    w = I.small_case(Pb.CCF, [1, 6, 1], 7, m=32, seed=5)
    p = Pb.Problem(Pb.CCF, [1, 6, 1], w.y, hilbert_m=32)
    ys = w.y
    D1 = p.d1_residuals(w.theta, w.lam, ys)[0, 0]
    D2 = p.d2_residuals(w.theta, w.lam, ys)[0, 0, 0]
    e = 1e-5 * np.maximum(1.0, np.abs(ys[0]))
    Rp = p.interior_residuals(w.theta, w.lam, ys + e)[0]
    Rm = p.interior_residuals(w.theta, w.lam, ys - e)[0]
    R0 = p.interior_residuals(w.theta, w.lam, ys)[0]
    fd1 = (Rp - Rm) / (2 * e)
    fd2 = (Rp - 2 * R0 + Rm) / e ** 2
    np.testing.assert_allclose(D1, fd1, rtol=1e-6, atol=1e-7 * np.max(np.abs(fd1)))
    np.testing.assert_allclose(D2, fd2, rtol=1e-3, atol=1e-4 * np.max(np.abs(fd2)))


def test_planted_wrong_diff_factor_breaks_closed_form_pin(monkeypatch):
    """Taylor.diff without the (a_i + 1) factor: the flat-residual pin must fail."""
    def wrong(self, i):
        K = self.K - 1
        c = {}
        from oracle.taylor import multi_indices
        for a in multi_indices(self.d, K):
            b = tuple(a[k] + (1 if k == i else 0) for k in range(self.d))
            c[a] = self.c[b]
        return Taylor(c, self.d, K)
    monkeypatch.setattr(Taylor, "diff", wrong)
    with pytest.raises(AssertionError):
        test_burgers_closed_forms_have_flat_residuals(3, 0.5)


def test_ccf_gradient_with_derivative_rows():
    """g = J~^T r~ stays the gradient of h with CCF d1 and d2 rows (complex step of h in theta,
    through the node values and the velocity series)."""
    w = I.small_case(Pb.CCF, [1, 6, 1], 8, m=32, seed=7)
    p = Pb.Problem(Pb.CCF, [1, 6, 1], w.y, hilbert_m=32, y_d1=w.y[:, :5], c_d1=0.6, y_d2=w.y[:, 2:6], c_d2=0.3)
    assert p.n_rows == p.n + 5 + 4 + 1
    J = gn.jacobian(p, w.theta, w.lam)
    g = J.T @ p.rows(w.theta, w.lam)
    x = np.concatenate([w.theta, [w.lam]]).astype(np.complex128)
    for j in [0, p.P // 2, p.P]:
        xc = x.copy()
        xc[j] += 1j * 1e-30
        r = p.rows(xc[:-1], xc[-1])
        dh = (0.5 * np.sum(r * r)).imag / 1e-30
        assert abs(dh - g[j]) <= 1e-10 * (abs(g[j]) + 1e-3 * np.max(np.abs(g)))


# ---------------------------------------------------------------------------
# the CCF velocity's Taylor series against a closed-form Hilbert pair, near the nodes too

def _node_distance(x, M):
    """Smallest distance from the points x to the circle nodes s_j, relative to 1 + |s_j|."""
    _, s = hilbert.nodes(M)
    return float(np.min(np.abs(np.asarray(x)[:, None] - s[None, :]) / (1.0 + np.abs(s[None, :]))))


@pytest.mark.parametrize("M", [16, 64])
def test_ccf_velocity_series_matches_a_hilbert_pair_near_nodes(M):
    """g(s) = s/(1+s^2) (Theta = s^2/(1+s^2)) has U(x) = x H[g](x) = -x/(1+x^2), which the discrete
    operator reproduces to rounding for M >= 8 (a trigonometric polynomial under the circle map).
    Its Taylor coefficients in x, differentiated analytically by sympy, pin velocity_series to
    order 4 at generic points and at points 1e-2, 1e-4 and 1e-6 (relative) from a node.  Near a node
    the k-th coefficient loses accuracy like eps / dist^(k+1) (the difference g_j - g(x), small
    there, carries an absolute rounding error that 1/(x - s_j)^(k+1) amplifies): the bound below says
    so, and the distances are reported in the assertion."""
    sp = pytest.importorskip("sympy")
    psi, s = hilbert.nodes(M)
    mid = np.tan(0.5 * (psi[[3, M // 2 - 2, M // 2 + 1, M - 5]] + np.pi / M))   # half-way between nodes
    generic = np.concatenate([np.linspace(-4.0, 4.0, 9), [0.37, 12.5, -130.0], mid])
    near = np.concatenate([s[[1, M // 3, M // 2]] + 1e-2 * (1 + np.abs(s[[1, M // 3, M // 2]])),
                           s[[2, M // 2 + 1]] - 1e-4 * (1 + np.abs(s[[2, M // 2 + 1]])),
                           s[[M // 4]] + 1e-6 * (1 + np.abs(s[[M // 4]]))])
    x = np.concatenate([generic, near])
    K = 4
    X = Taylor.variable(x, 0, 1, K)
    gX = X / (X * X + 1.0)
    g_nodes = s / (1.0 + s * s)
    U = hilbert.velocity_series(X, gX, g_nodes, M)
    t = sp.symbols("t")
    f = -t / (1 + t * t)
    coef = [sp.lambdify(t, sp.diff(f, t, k) / sp.factorial(k), "numpy") for k in range(K + 1)]
    dist = np.min(np.abs(x[:, None] - s[None, :]) / (1.0 + np.abs(s[None, :])), axis=1)
    for k in range(K + 1):
        want = np.asarray(coef[k](x), dtype=np.float64)
        got = U.c[(k,)]
        bound = 1e-14 * np.sqrt(M) * (1.0 + np.abs(x)) ** 2 * (1.0 + dist ** (-(k + 1)))
        err = np.abs(got - want)
        assert np.all(err <= bound), (k, float(np.max(err / bound)), float(np.min(dist)))
    # points at least 0.04 (relative) from every node keep 1e-11 through order 4
    far = dist >= 0.04
    assert np.count_nonzero(far) >= 6
    ferr = max(float(np.max(np.abs(U.c[(k,)][far] - np.asarray(coef[k](x[far]), dtype=np.float64))))
               for k in range(K + 1))
    assert ferr <= 1e-11, ferr


def test_ccf_derivative_test_points_stay_away_from_nodes():
    """The GPU parity cases of the CCF derivative rows (M = 32) keep their points at least 1e-2
    (relative) from every node, where both sides' orders of summation agree to far below 1e-12."""
    from paper_2509_14185_gb300 import inputs as I
    w = I.with_derivative_batches(I.small_case(I.CCF, [1, 40, 40, 1], 60, seed=13, m=32), 11, 9)
    assert _node_distance(w.y_d1[0], 32) > 1e-2
    assert _node_distance(w.y_d2[0], 32) > 1e-2
