"""Pin of the oracle's row weights to the paper's training loss (Methods, "Training Loss").

The oracle assembles weighted rows r~ and defines h = 1/2 |r~|^2.  The paper defines the loss
term by term:

  L_d0   = 1/(N_d0 N_E)     sum_{(y, rho) in Y0} rho sum_k R_k(y)^2
  L_d1   = 1/(N_d1 N_E d)   sum_{(y, rho) in Y1} rho sum_k sum_i (d_i R_k(y))^2
  L_d2   = 1/(N_d2 N_E d^2) sum_{(y, rho) in Y2} rho sum_k sum_{i,j} (d_i d_j R_k(y))^2
  L_eq   = L_d0 + c_d1 L_d1 + c_d2 L_d2
  L_data = c_norm (Phi_A0(y_norm) - C)^2 + c_inf sum_{Y_inf} Phi_A0(y)^2
           (+ the wall term (c_bnd / N_b) sum_b Psi(y_b)^2 and relu bound terms, the
           constraints the paper says some problems add)
  L      = L_eq + L_data.

Here that sum is written out with plain Python loops over points, equations and derivative
indices from the oracle's unweighted quantities (R_k values, their y-derivatives, the wall,
decay, bound and normalisation values), never through `Problem.rows`.  The test asserts
h == L to 1e-14 with non-uniform rho, c_bnd != 1, c_norm_w != 1, c_inf != 1, c_relu != 1,
c_d1 != 1, c_d2 != 1, for N_E = 1, 2 and 3.  Planted mistakes (each a faithful emulation of what
a wrong row weight would output: a dropped factor 2, 1/N instead of 1/(N N_E), rho ignored, a
wall weight without the 1/N_b, a derivative weight without its 1/d) must each fail the pin.
"""
import numpy as np
import pytest

from oracle import problems as Pb
from paper_2509_14185_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

CASES = [
    (Pb.BURGERS, [1, 6, 5, 1], 9, 0),
    (Pb.CCF, [1, 6, 5, 1], 9, 0),
    (Pb.IPM, [2, 5, 4, 2], 8, 4),
    (Pb.BOUSSINESQ, [2, 5, 4, 3], 8, 4),
]

W = dict(c_bnd=2.75, c_norm_w=0.35, c_inf=1.6, c_relu=0.45, c_d1=0.3, c_d2=0.07)


def make_problem(eq, widths, n, nb, derivative_losses=True):
    w = I.small_case(eq, widths, n, n_bnd=nb, seed=17, m=16)
    d = w.d
    rho = 0.25 + 3.75 * I.uniform(901, n)                   # non-uniform point weights
    far = 10.0 ** (1.0 + 1.5 * I.uniform(902, 3))
    if d == 1:
        y_inf = far.reshape(1, -1)
        y_relu = (0.3 + I.uniform(903, 4)).reshape(1, -1)
    else:
        a = 0.5 * np.pi * I.uniform(904, 3)
        y_inf = np.stack([far * np.cos(a), far * np.sin(a)])
        rr, aa = 0.3 + I.uniform(905, 4), 0.5 * np.pi * I.uniform(906, 4)
        y_relu = np.stack([rr * np.cos(aa), rr * np.sin(aa)])
    kw = dict(y_inf=y_inf, y_relu=y_relu, relu_bound=0.0, relu_sign=1)
    if derivative_losses:
        kw.update(y_d1=w.y[:, :4], rho_d1=0.5 + I.uniform(907, 4), y_d2=w.y[:, 2:5], rho_d2=0.5 + I.uniform(908, 3))
    p = Pb.Problem(eq, widths, w.y, w.y_bnd if nb else None, rho, y_norm=w.y_norm, c_norm=w.c_norm,
                   hilbert_m=16, **W, **kw)
    return w, p


def paper_loss(p, theta, lam):
    """L_train written term by term from the printed definitions (loops, no row vector)."""
    R = p.interior_residuals(theta, lam)                  # N_E arrays over the points
    N, NE, d = p.n, p.ne, p.d
    L_d0 = 0.0
    for i in range(N):
        s = 0.0
        for k in range(NE):
            s += R[k][i] ** 2
        L_d0 += p.rho[i] * s
    L_d0 /= N * NE
    L_d1 = 0.0
    if p.n_d1:
        D1 = p.d1_residuals(theta, lam)                   # (N_E, d, n)
        for i in range(p.n_d1):
            s = 0.0
            for k in range(NE):
                for a in range(d):
                    s += D1[k][a][i] ** 2
            L_d1 += p.rho_d1[i] * s
        L_d1 /= p.n_d1 * NE * d
    L_d2 = 0.0
    if p.n_d2:
        D2 = p.d2_residuals(theta, lam)                   # (N_E, d, d, n)
        for i in range(p.n_d2):
            s = 0.0
            for k in range(NE):
                for a in range(d):
                    for b in range(d):
                        s += D2[k][a][b][i] ** 2
            L_d2 += p.rho_d2[i] * s
        L_d2 /= p.n_d2 * NE * d * d
    L_eq = L_d0 + p.c_d1 * L_d1 + p.c_d2 * L_d2
    L_data = p.c_norm_w * (p.norm_value(theta, lam) - p.c_norm) ** 2
    for v in p.inf_values(theta, lam):
        L_data += p.c_inf * v ** 2
    for v in p.relu_values(theta, lam):
        L_data += p.c_relu * v ** 2
    if p.nb:
        wall = 0.0
        for v in p.wall_values(theta, lam):
            wall += v ** 2
        L_data += p.c_bnd / p.nb * wall
    return L_eq + L_data


def check(p, theta, lam):
    h = p.loss(theta, lam)
    L = paper_loss(p, theta, lam)
    return abs(h - L) <= 1e-14 * abs(L), h, L


@pytest.mark.parametrize("eq,widths,n,nb", CASES)
def test_rows_reproduce_the_paper_loss(eq, widths, n, nb):
    w, p = make_problem(eq, widths, n, nb)
    assert len(set(np.round(p.rho, 6))) == p.n                # really non-uniform
    assert p.nrelu and np.any(p.relu_values(w.theta, w.lam) != 0.0)   # some bound rows active
    ok, h, L = check(p, w.theta, w.lam)
    assert ok, (h, L)
    # every part of the loss has its rows
    assert p.n_rows == (p.n * p.ne + p.n_d1 * p.ne * p.d + p.n_d2 * p.ne * p.d ** 2 + p.nb + p.ninf
                        + p.nrelu + 1)


@pytest.mark.parametrize("eq,widths,n,nb", CASES[2:])
def test_rows_reproduce_the_paper_loss_without_derivative_batches(eq, widths, n, nb):
    w, p = make_problem(eq, widths, n, nb, derivative_losses=False)
    ok, h, L = check(p, w.theta, w.lam)
    assert ok, (h, L)


# ---------------------------------------------------------------------------
# planted mistakes (CPU only): each wrong weighting must fail the pin.  A mistake is
# planted by wrapping Problem.rows so that it returns what the mistaken assembly would
# return; the pin (paper_loss) is left untouched.

def _segments(p):
    """Row ranges of the parts, in the oracle's documented order."""
    n0 = p.n * p.ne
    n1 = p.n_d1 * p.ne * p.d
    n2 = p.n_d2 * p.ne * p.d ** 2
    s = {"d0": (0, n0), "d1": (n0, n0 + n1), "d2": (n0 + n1, n0 + n1 + n2)}
    o = n0 + n1 + n2
    s["wall"] = (o, o + p.nb)
    return s


def _plant(monkeypatch, mutate):
    orig = Pb.Problem.rows

    def rows(self, theta, lam):
        return mutate(self, orig(self, theta, lam).copy())
    monkeypatch.setattr(Pb.Problem, "rows", rows)


def _dropped_two(p, r):
    return r / np.sqrt(2.0)


def _one_over_n(p, r):
    a, b = _segments(p)["d0"]
    r[a:b] *= np.sqrt(p.ne)
    return r


def _rho_ignored(p, r):
    a, b = _segments(p)["d0"]
    r[a:b] /= np.repeat(np.sqrt(p.rho), p.ne)
    return r


def _wall_without_mean(p, r):
    a, b = _segments(p)["wall"]
    r[a:b] *= np.sqrt(p.nb)
    return r


def _d1_without_dimension(p, r):
    a, b = _segments(p)["d1"]
    r[a:b] *= np.sqrt(p.d)
    return r


def _d2_single_mixed_pair(p, r):
    # counting the mixed pair (1, 2) once instead of twice: drop the (2, 1) rows
    a, b = _segments(p)["d2"]
    blk = r[a:b].reshape(p.n_d2, p.ne, p.d, p.d)
    blk[:, :, 1, 0] = 0.0
    r[a:b] = blk.reshape(-1)
    return r


@pytest.mark.parametrize("mutate,cases", [
    (_dropped_two, CASES),
    (_one_over_n, CASES[2:]),          # needs N_E > 1
    (_rho_ignored, CASES),
    (_wall_without_mean, CASES[2:]),   # needs a wall
    (_d1_without_dimension, CASES[2:]),  # needs d > 1
    (_d2_single_mixed_pair, CASES[2:]),
])
def test_planted_weight_mistakes_break_the_pin(monkeypatch, mutate, cases):
    probs = [make_problem(*c) for c in cases]
    _plant(monkeypatch, mutate)
    for w, p in probs:
        ok, h, L = check(p, w.theta, w.lam)
        assert not ok, (mutate.__name__, h, L)
