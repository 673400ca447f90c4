"""Pins for the data loss's decay rows (Methods, "Training Loss": the normalised field
Phi_{A0} must vanish at a set of points Y_inf far from the origin, weight c_inf).

* Constant network (every weight zero, output bias b): each field is the ansatz envelope
  times b, Phi_A = s_A(y) b q^{-k_A} with q = (1 + |y|^2)^{-1/(2(1+lambda))}, written out
  here from that definition for each equation's normalised field (Burgers U, CCF Theta,
  IPM P, Boussinesq Omega: odd, even, even, odd; k = lambda, lambda, lambda, -1).  The
  decay rows must be sqrt(2 c_inf) times those values, between the wall rows and the
  normalisation row.
* A decay point is a normalisation row with target 0 and the same weight (except for
  Boussinesq, whose normalisation row is a derivative): the two assemblies agree on a
  trained-looking random network.
* g = J~^T r~ stays the gradient of h with decay rows (complex step of h, no Jacobian code).
"""
import numpy as np
import pytest

from oracle import gn
from oracle import problems as Pb
from paper_2509_14185_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

CASES = [(Pb.BURGERS, [1, 5, 1]), (Pb.CCF, [1, 5, 1]), (Pb.IPM, [2, 5, 2]), (Pb.BOUSSINESQ, [2, 5, 3])]


def far_points(d, n, seed):
    rng = np.random.default_rng(seed)
    r = 10.0 ** rng.uniform(1.0, 3.0, n)
    if d == 1:
        return (r * rng.choice([-1.0, 1.0], n)).reshape(1, n)
    a = rng.uniform(0.0, np.pi / 2, n)
    return np.stack([r * np.cos(a), r * np.sin(a)])


def closed_form_field0(eq, y, lam, b):
    """Phi_{A0} of the constant network NN = b, from the ansatz definition."""
    u = 1.0 + np.sum(y * y, axis=0)
    q = u ** (-1.0 / (2.0 * (1.0 + lam)))
    if eq == Pb.BURGERS:
        return (y[0] / np.sqrt(u)) * b * q ** (-lam)
    if eq == Pb.CCF:
        return (y[0] ** 2 / u) * b * q ** (-lam)
    if eq == Pb.IPM:
        return b * q ** (-lam)
    return (y[0] / np.sqrt(u)) * b * q      # Boussinesq Omega, k = -1


@pytest.mark.parametrize("eq,widths", CASES)
def test_decay_rows_of_constant_network(eq, widths):
    w = I.small_case(eq, widths, 7, n_bnd=3, m=16)
    yinf = far_points(w.d, 5, 3)
    c_inf = 0.7
    p = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=w.y_norm, hilbert_m=16, y_inf=yinf, c_inf=c_inf)
    theta = np.zeros(p.P)
    b = np.array([1.3, -0.4, 0.9])[: widths[-1]]
    theta[-widths[-1]:] = b
    lam = 0.37
    r = p.rows(theta, lam)
    assert len(r) == p.n_rows == p.n * p.ne + p.nb + 5 + 1
    lo = p.n * p.ne + p.nb
    want = np.sqrt(2.0 * c_inf) * closed_form_field0(eq, yinf, lam, b[0])
    np.testing.assert_allclose(r[lo:lo + 5], want, rtol=1e-13, atol=1e-300)
    # the other rows are those of the problem without decay points, in place
    p0 = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=w.y_norm, hilbert_m=16)
    r0 = p0.rows(theta, lam)
    np.testing.assert_array_equal(r[:lo], r0[:lo])
    assert r[-1] == r0[-1]
    # and the loss gains exactly c_inf sum Phi^2
    assert p.loss(theta, lam) == pytest.approx(p0.loss(theta, lam) + c_inf * np.sum(want ** 2 / (2 * c_inf)),
                                               rel=1e-14)


@pytest.mark.parametrize("eq,widths", CASES[:3])
def test_decay_row_is_a_zero_target_normalisation_row(eq, widths):
    w = I.small_case(eq, widths, 6, n_bnd=2, m=16, seed=4)
    yinf = far_points(w.d, 3, 8)
    p = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=w.y_norm, hilbert_m=16, y_inf=yinf, c_inf=2.5)
    r = p.rows(w.theta, w.lam)
    lo = p.n * p.ne + p.nb
    for k in range(3):
        yn = tuple(yinf[:, k]) + ((0.0,) if w.d == 1 else ())
        pn = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=yn, c_norm=0.0, c_norm_w=2.5, hilbert_m=16)
        assert r[lo + k] == pytest.approx(pn.rows(w.theta, w.lam)[-1], rel=1e-14, abs=1e-300)


@pytest.mark.parametrize("eq,widths", [(Pb.CCF, [1, 6, 1]), (Pb.BOUSSINESQ, [2, 5, 3])])
def test_gradient_with_decay_rows(eq, widths):
    w = I.small_case(eq, widths, 10, n_bnd=4, m=32)
    p = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=w.y_norm, hilbert_m=32, y_inf=far_points(w.d, 4, 1),
                   c_inf=0.5)
    J = gn.jacobian(p, w.theta, w.lam)
    g = J.T @ p.rows(w.theta, w.lam)
    x = np.concatenate([w.theta, [w.lam]]).astype(np.complex128)
    h = 1e-30
    for j in [0, p.P // 2, p.P]:
        xc = x.copy()
        xc[j] += 1j * h
        r = p.rows(xc[:-1], xc[-1])
        dh = (0.5 * np.sum(r * r)).imag / h
        assert abs(dh - g[j]) <= 1e-11 * (abs(g[j]) + 1e-3 * np.max(np.abs(g)))


# the normalisation constraint on another field, or on a derivative (Methods, "Training Loss":
# constraints may act on more than one field or on derivatives of a field)

def closed_form_field(eq, f, y, lam, b):
    """Field f of the constant network NN = b from the ansatz: s_A b q^{-k_A} with the
    parity classes (odd: s = y1 / sqrt(u), even: s = 1) and exponents of each equation."""
    u = 1.0 + np.sum(y * y, axis=0)
    q = u ** (-1.0 / (2.0 * (1.0 + lam)))
    odd = y[0] / np.sqrt(u)
    if eq == Pb.IPM:
        return [b * q ** (-lam), odd * b * q ** (-(1.0 + 2.0 * lam))][f]
    return [odd * b * q, b * q ** (-(lam - 1.0)), odd * b * q ** (-(1.0 + 2.0 * lam))][f]


@pytest.mark.parametrize("eq,widths", [(Pb.IPM, [2, 4, 2]), (Pb.BOUSSINESQ, [2, 4, 3])])
def test_normalisation_on_each_field(eq, widths):
    w = I.small_case(eq, widths, 5, n_bnd=2, m=16)
    lam, yn, cn, cw = 0.41, (0.7, 1.3), 0.25, 1.7
    b = np.array([1.3, -0.4, 0.9])[: widths[-1]]
    for f in range(widths[-1]):
        p = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=yn, c_norm=cn, c_norm_w=cw, norm_field=f, norm_deriv=0,
                       y_inf=far_points(2, 3, 2), c_inf=0.6)
        theta = np.zeros(p.P)
        theta[-widths[-1]:] = b
        r = p.rows(theta, lam)
        phi = closed_form_field(eq, f, np.array(yn).reshape(2, 1), lam, b[f])[0]
        assert r[-1] == pytest.approx(np.sqrt(2.0 * cw) * (phi - cn), rel=1e-13)
        # the decay rows constrain the same field
        lo = p.n * p.ne + p.nb
        want = np.sqrt(2.0 * 0.6) * closed_form_field(eq, f, p.y_inf, lam, b[f])
        np.testing.assert_allclose(r[lo:lo + 3], want, rtol=1e-13)


@pytest.mark.parametrize("eq,widths,f", [(Pb.BURGERS, [1, 6, 1], 0), (Pb.IPM, [2, 6, 2], 1),
                                         (Pb.BOUSSINESQ, [2, 6, 3], 1)])
def test_normalisation_derivative_is_d_dy1_of_the_value(eq, widths, f):
    w = I.small_case(eq, widths, 5, n_bnd=2, m=16, seed=9)
    yn = (0.8, 0.6)
    kw = dict(c_norm=0.0, c_norm_w=0.5, norm_field=f)
    p = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=yn, norm_deriv=1, **kw)
    d = p.rows(w.theta, w.lam)[-1]
    h = 1e-5
    vals = []
    for s in (1.0, -1.0):
        ys = (yn[0] + s * h, yn[1])
        pv = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=ys, norm_deriv=0, **kw)
        vals.append(pv.rows(w.theta, w.lam)[-1])
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(d - fd) <= 1e-7 * max(1.0, abs(d))
    # and the defaults are the equation's own constraint (Boussinesq: d1 Omega; others: the value)
    p0 = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=yn)
    assert p0.norm_field == 0 and p0.norm_deriv == (1 if eq == Pb.BOUSSINESQ else 0)


# planted mistakes (on the CPU only): each pin above must fail when the oracle is wrong

def test_planted_wrong_field_breaks_decay_pin(monkeypatch):
    """Decay rows built from field 1 instead of the constrained field 0."""
    def wrong(self, theta, lam):
        return self.fields(theta, lam, self.y_inf)[min(1, N_FIELDS_OF[self.eq] - 1)].v
    monkeypatch.setattr(Pb.Problem, "inf_values", wrong)
    with pytest.raises(AssertionError):
        test_decay_rows_of_constant_network(Pb.IPM, [2, 5, 2])


def test_planted_missing_weight_breaks_decay_pin(monkeypatch):
    """The decay rows without their sqrt(2 c_inf) weight (rows of c_inf / 2 times the loss)."""
    orig = Pb.Problem.rows

    def wrong(self, theta, lam):
        r = orig(self, theta, lam).copy()
        lo = self.n * self.ne + self.nb
        r[lo:lo + self.ninf] /= np.sqrt(2.0 * self.c_inf)
        return r
    monkeypatch.setattr(Pb.Problem, "rows", wrong)
    with pytest.raises(AssertionError):
        test_decay_rows_of_constant_network(Pb.BURGERS, [1, 5, 1])


def test_planted_value_for_derivative_breaks_normalisation_pin(monkeypatch):
    """A normalisation row that ignores norm_deriv (always the value)."""
    def wrong(self, theta, lam):
        ys = np.array(self.y_norm[:self.d], dtype=np.float64).reshape(self.d, 1)
        return self.fields(theta, lam, ys)[self.norm_field].v[0]
    monkeypatch.setattr(Pb.Problem, "norm_value", wrong)
    with pytest.raises(AssertionError):
        test_normalisation_derivative_is_d_dy1_of_the_value(Pb.IPM, [2, 6, 2], 1)


N_FIELDS_OF = {Pb.BURGERS: 1, Pb.CCF: 1, Pb.IPM: 2, Pb.BOUSSINESQ: 3}


# bound constraints: relu(s (Phi_A0(y) - b)) before squaring (Methods, "Training Loss")

@pytest.mark.parametrize("eq,widths", CASES)
@pytest.mark.parametrize("sign", [1, -1])
def test_relu_bound_rows_of_constant_network(eq, widths, sign):
    w = I.small_case(eq, widths, 6, n_bnd=2, m=16)
    yb = far_points(w.d, 6, 5) * 0.01            # points near the origin: field values O(1)
    b = np.array([1.3, -0.4, 0.9])[: widths[-1]]
    lam = 0.37
    phi = closed_form_field0(eq, yb, lam, b[0])
    bound = float(np.median(phi))                 # half the points on each side
    p = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=w.y_norm, hilbert_m=16, y_inf=far_points(w.d, 2, 1),
                   y_relu=yb, c_relu=0.8, relu_bound=bound, relu_sign=sign)
    theta = np.zeros(p.P)
    theta[-widths[-1]:] = b
    r = p.rows(theta, lam)
    lo = p.n * p.ne + p.nb + p.ninf
    want = np.sqrt(1.6) * np.maximum(sign * (phi - bound), 0.0)
    np.testing.assert_allclose(r[lo:lo + 6], want, rtol=1e-13, atol=1e-300)
    assert np.sum(want > 0) >= 2 and np.sum(want == 0) >= 2
    assert len(r) == p.n_rows and r[-1] == Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=w.y_norm,
                                                      hilbert_m=16).rows(theta, lam)[-1]


@pytest.mark.parametrize("eq,widths", [(Pb.BURGERS, [1, 6, 1]), (Pb.IPM, [2, 5, 2])])
def test_relu_rows_gradient_and_inactive_rows(eq, widths):
    w = I.small_case(eq, widths, 8, n_bnd=2, m=16, seed=2)
    yb = far_points(w.d, 6, 9) * 0.02
    p0 = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=w.y_norm, hilbert_m=16, y_relu=yb)
    vals = p0.fields(w.theta, w.lam, yb)[0].v
    p = Pb.Problem(eq, widths, w.y, w.y_bnd, y_norm=w.y_norm, hilbert_m=16, y_relu=yb, c_relu=0.5,
                   relu_bound=float(np.median(vals)), relu_sign=1)
    J = gn.jacobian(p, w.theta, w.lam)
    r = p.rows(w.theta, w.lam)
    lo = p.n * p.ne + p.nb + p.ninf
    inactive = r[lo:lo + 6] == 0.0
    assert inactive.any() and (~inactive).any()
    assert np.all(J[lo:lo + 6][inactive] == 0.0)          # no gradient through an inactive bound
    g = J.T @ r
    x = np.concatenate([w.theta, [w.lam]]).astype(np.complex128)
    for j in [0, p.P // 2, p.P]:
        xc = x.copy()
        xc[j] += 1j * 1e-30
        rc = p.rows(xc[:-1], xc[-1])
        dh = (0.5 * np.sum(rc * rc)).imag / 1e-30
        assert abs(dh - g[j]) <= 1e-11 * (abs(g[j]) + 1e-3 * np.max(np.abs(g)))
