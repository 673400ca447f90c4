"""Pins for the oracle's Gauss-Newton machinery and the residual symmetries.

* Cholesky: textbook factorisation vs numpy's LAPACK routine and the
  reconstruction L L^T = A; non-SPD input is reported, not factorised.
* GN step on a linear least-squares problem r(x) = A x - b: with damping
  gamma -> 0 one step lands on the normal-equations solution, the line search
  accepts alpha = 1 and the Levenberg-Marquardt ratio is exactly 1.
* g = J~^T r~ is the gradient of h = |r~|^2 / 2 (checked by central
  differences of h, which uses no Jacobian code).
* Odd/even symmetry in y1 of every residual, as fixed by the parity of the
  fields (Methods, "Solution Modeling").
* Planted mistakes: the pins above fail when a typical error is introduced
  into the oracle (monkeypatched on the CPU only).
"""
import numpy as np
import pytest
import sympy as sp

from oracle import gn
from oracle import problems as Pb
from paper_2509_14185_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_cholesky_vs_library():
    rng = np.random.default_rng(3)
    for n in [1, 2, 7, 40]:
        B = rng.standard_normal((n + 3, n))
        A = B.T @ B + 0.1 * np.eye(n)
        L, ok = gn.cholesky(A)
        assert ok
        np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(L @ L.T, A, rtol=1e-13, atol=1e-13)
        b = rng.standard_normal(n)
        x = gn.cholesky_solve(L, b)
        np.testing.assert_allclose(A @ x, b, rtol=1e-11, atol=1e-12)
    A = np.array([[1.0, 2.0], [2.0, 1.0]])
    assert not gn.cholesky(A)[1]


def test_damped_solve_escalates_gamma():
    A = -np.eye(3)
    delta, gamma, retries, ok = gn.damped_solve(A, np.ones(3), 0.5)
    assert ok and retries == 1 and gamma == 5.0
    np.testing.assert_allclose(delta, np.ones(3) / 4.0)
    _, _, retries, ok = gn.damped_solve(-1e9 * np.eye(3), np.ones(3), 1.0)
    assert not ok and retries == gn.MAX_CHOL_RETRIES


def test_gn_step_linear_least_squares():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 6))
    b = rng.standard_normal(30)
    x0 = rng.standard_normal(6)
    x1, gamma, info = gn.gn_step_generic(lambda x: A @ x - b, lambda x: A, x0, 1e-14)
    xs = np.linalg.lstsq(A, b, rcond=None)[0]
    np.testing.assert_allclose(x1, xs, rtol=1e-10, atol=1e-12)
    assert info["alpha"] == 1.0 and info["status"] == gn.STEP_OK
    assert abs(info["rho"] - 1.0) < 1e-8
    assert gamma == pytest.approx(1e-14 * 2 / 3)


def test_gn_step_no_decrease_keeps_point():
    # r(x) = x^2 - 1 at x = 0: J = 0, so G + gamma I gives delta = 0; with a
    # gradient of zero the Armijo test is met at alpha = 1 with equality.
    x1, gamma, info = gn.gn_step_generic(lambda x: np.array([1e300 * x[0] ** 2 + 1.0]),
                                         lambda x: np.array([[1.0]]), np.array([1.0]), 1.0)
    assert info["status"] == gn.WARN_NO_DECREASE
    assert x1[0] == 1.0 and gamma == 10.0


@pytest.mark.parametrize("eq,widths", [(Pb.CCF, [1, 6, 6, 1]), (Pb.IPM, [2, 5, 5, 2]),
                                       (Pb.BOUSSINESQ, [2, 5, 5, 3])])
def test_gradient_is_grad_of_loss(eq, widths):
    w = I.small_case(eq, widths, 12, n_bnd=4, m=32)
    p = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=w.y_norm, hilbert_m=32)
    J = gn.jacobian(p, w.theta, w.lam)
    g = J.T @ p.rows(w.theta, w.lam)
    x = np.concatenate([w.theta, [w.lam]]).astype(np.complex128)
    h = 1e-30
    for j in [1, p.P // 3, p.P]:
        # complex step of the scalar loss h = r.r/2 (no Jacobian code involved)
        xc = x.copy()
        xc[j] += 1j * h
        r = p.rows(xc[:-1], xc[-1])
        dh = (0.5 * np.sum(r * r)).imag / h
        assert abs(dh - g[j]) <= 1e-11 * (abs(g[j]) + 1e-3 * np.max(np.abs(g)))
        # and a loose central difference
        e = 1e-6 * max(1.0, abs(x[j].real))
        xp, xm = x.real.copy(), x.real.copy()
        xp[j] += e
        xm[j] -= e
        fd = (p.loss(xp[:-1], xp[-1]) - p.loss(xm[:-1], xm[-1])) / (2 * e)
        assert abs(fd - g[j]) <= 1e-5 * abs(g[j]) + 1e-6 * np.max(np.abs(g))


PARITY = {Pb.BURGERS: [-1], Pb.CCF: [1], Pb.IPM: [1, -1], Pb.BOUSSINESQ: [-1, 1, -1]}


@pytest.mark.parametrize("eq,widths", [(Pb.BURGERS, [1, 6, 1]), (Pb.CCF, [1, 6, 1]),
                                       (Pb.IPM, [2, 6, 2]), (Pb.BOUSSINESQ, [2, 6, 3])])
def test_residual_parity_in_y1(eq, widths):
    w = I.small_case(eq, widths, 16, m=64)
    p = Pb.Problem(eq, widths, w.y, hilbert_m=64)
    ys = w.y.copy()
    ym = ys.copy()
    ym[0] = -ym[0]
    R = p.interior_residuals(w.theta, w.lam, ys)
    Rm = p.interior_residuals(w.theta, w.lam, ym)
    for k, s in enumerate(PARITY[eq]):
        np.testing.assert_allclose(Rm[k], s * R[k], rtol=1e-11, atol=1e-12 * np.max(np.abs(R[k])))


def test_boussinesq_norm_row_is_d1_omega_at_origin():
    widths = [2, 5, 3]
    w = I.small_case(Pb.BOUSSINESQ, widths, 4)
    p = Pb.Problem(Pb.BOUSSINESQ, widths, w.y, y_norm=(0.0, 0.0))
    # d1 Omega(0,0) = NN_Omega(q=1, beta=0): evaluate the network by hand
    (W0, b0), (W1, b1) = p.layers(w.theta)
    nn = W1 @ np.tanh(W0 @ np.array([1.0, 0.0]) + b0) + b1
    assert p.norm_value(w.theta, w.lam) == pytest.approx(nn[0], rel=1e-14)


# ---------------------------------------------------------------------------
# planted mistakes: each pin must fail when the oracle is wrong
# ---------------------------------------------------------------------------

def test_planted_wrong_theta_exponent_breaks_lambda_inference(monkeypatch):
    from tests import test_oracle_pde_reduction as T
    orig = Pb.residual_boussinesq

    def wrong(lam, *a):
        R = orig(lam, *a)
        Th = a[5]
        return [R[0], R[1] - Th, R[2]]   # k_theta = lambda instead of lambda - 1
    monkeypatch.setattr(Pb, "residual_boussinesq", wrong)
    with pytest.raises(AssertionError):
        T.test_boussinesq_lambda_inference_rule_from_paper()
    with pytest.raises(AssertionError):
        T.test_boussinesq_reduction()


def test_planted_sign_error_breaks_ipm_reduction(monkeypatch):
    from tests import test_oracle_pde_reduction as T
    orig = Pb.residual_ipm

    def wrong(lam, y1, y2, P, P_1, P_2, Psi_1, Psi_2, Psi_11, Psi_22):
        return orig(lam, y1, y2, P, P_1, P_2, -Psi_1, Psi_2, Psi_11, Psi_22)  # u2 = +d1 psi
    monkeypatch.setattr(Pb, "residual_ipm", wrong)
    with pytest.raises(AssertionError):
        T.test_ipm_reduction()


def test_planted_wrong_hilbert_constant_breaks_pair(monkeypatch):
    from oracle import hilbert
    from tests import test_oracle_closed_forms as T
    orig = hilbert.nodes

    def shifted(M):
        psi, s = orig(M)
        return psi, s * 1.01
    monkeypatch.setattr(hilbert, "nodes", shifted)
    with pytest.raises(AssertionError):
        T.test_ccf_velocity_factorised_pair(8)


def test_planted_transposed_jacobian_breaks_linear_step():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((6, 6))
    b = rng.standard_normal(6)
    x1, _, _ = gn.gn_step_generic(lambda x: A @ x - b, lambda x: A.T, np.zeros(6), 1e-14)
    assert np.max(np.abs(x1 - np.linalg.solve(A, b))) > 1e-3


# ---------------------------------------------------------------------------
# the paper's EMA rank-1 optimiser (Methods, "Second-order Optimizer")
# ---------------------------------------------------------------------------
def test_rank1_estimate_is_unbiased_exactly():
    """E[u u^T] = J^T J for u = J^T v with independent +-1 signs: averaging over all 2^R
    sign vectors of a small J gives J^T J to rounding."""
    import itertools
    rng = np.random.default_rng(3)
    J = rng.standard_normal((6, 4))
    acc = np.zeros((4, 4))
    for bits in itertools.product([-1.0, 1.0], repeat=6):
        u = gn.rank1_estimate(J, np.array(bits))
        acc += np.outer(u, u)
    acc /= 2 ** 6
    assert np.max(np.abs(acc - J.T @ J)) <= 1e-13 * np.max(np.abs(J.T @ J))


def test_mg_coefficients_minimise_the_model():
    """(alpha, mu) from the 2 x 2 normal equations is the minimiser of the quadratic
    g.d + 1/2 d.C.d over the plane spanned by Delta and v (checked against a dense grid
    refinement and by the zero gradient)."""
    rng = np.random.default_rng(5)
    B = rng.standard_normal((7, 7))
    C = B.T @ B + 0.1 * np.eye(7)
    g = rng.standard_normal(7)
    D, v = rng.standard_normal(7), rng.standard_normal(7)
    a, m = gn.mg_coefficients(D @ C @ D, D @ C @ v, v @ C @ v, g @ D, g @ v, True)

    def model(a, m):
        d = a * D + m * v
        return g @ d + 0.5 * d @ C @ d

    f0 = model(a, m)
    for da, dm in [(1e-3, 0), (-1e-3, 0), (0, 1e-3), (0, -1e-3), (1e-3, 1e-3), (-1e-3, 1e-3)]:
        assert model(a + da, m + dm) > f0
    h = 1e-6
    assert abs((model(a + h, m) - model(a - h, m)) / (2 * h)) < 1e-6
    assert abs((model(a, m + h) - model(a, m - h)) / (2 * h)) < 1e-6
    a1, m1 = gn.mg_coefficients(D @ C @ D, 0.0, 1.0, g @ D, 0.0, False)
    assert m1 == 0.0 and abs(a1 + (g @ D) / (D @ C @ D)) < 1e-15


def test_ema_step_with_exact_curvature_is_the_damped_gn_step():
    """Special case: when the average already equals the exact G (beta = 1 keeps it) and there
    is no previous update, Delta = -(G + gamma I)^{-1} g and the closed-form alpha is exactly 1
    (Delta.C.Delta = -g.Delta for C = G + gamma I), so the step is the plain damped GN step."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((12, 5))
    b = rng.standard_normal(12)

    def rows_fn(x):
        return A @ x - b

    def jac_fn(x):
        return A

    x0 = np.zeros(5)
    G = A.T @ A
    gamma = 1e-3
    xn, gam, Gn, vn, info = gn.ema_step_generic(rows_fn, jac_fn, x0, gamma, G, np.zeros(5), np.ones(12), 1.0,
                                                 False)
    assert abs(info["alpha"] - 1.0) < 1e-12 and info["mu"] == 0.0
    step = -np.linalg.solve(G + gamma * np.eye(5), A.T @ (A @ x0 - b))
    assert np.max(np.abs(xn - (x0 + step))) <= 1e-12 * np.max(np.abs(step))
    assert np.array_equal(Gn, G) and np.max(np.abs(vn - step)) <= 1e-12 * np.max(np.abs(step))


def test_ema_step_first_step_uses_the_rank1_sample_and_reaches_least_squares():
    """On a linear least-squares problem the EMA optimiser starts its average from the first
    rank-1 sample, never increases the objective (the closed-form step minimises the model,
    which is exact for a linear residual) and reaches the least-squares minimum (closed form)."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((30, 6))
    b = rng.standard_normal(30)

    def rows_fn(x):
        return A @ x - b

    def jac_fn(x):
        return A

    s = I.signs(4, 30)
    assert set(np.unique(s)) == {-1.0, 1.0}
    xs = np.linalg.lstsq(A, b, rcond=None)[0]
    hmin = 0.5 * float((A @ xs - b) @ (A @ xs - b))
    x = np.zeros(6)
    G = np.zeros((6, 6))
    v = np.zeros(6)
    gamma = 1.0
    for k in range(40):
        sk = I.signs(4, 30, 30 * k)
        x, gamma, Gn, v, info = gn.ema_step_generic(rows_fn, jac_fn, x, gamma, G, v, sk, 0.9, k == 0)
        u = A.T @ sk
        expect = np.outer(u, u) if k == 0 else 0.9 * G + (1.0 - 0.9) * np.outer(u, u)
        assert np.array_equal(Gn, expect)
        G = Gn
        assert info["loss_after"] <= info["loss_before"] * (1 + 1e-12)
    assert abs(info["loss_after"] - hmin) <= 1e-9 * hmin
