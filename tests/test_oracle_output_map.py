"""Pins for the exponential output map (Methods, "Solution Modeling": the last activation is
exponential or exponential-adjacent; this project's default reading is linear, exp a flag).

* Constant network (every weight zero, output bias b): NN = exp(b), so each field is the
  ansatz envelope times exp(b), written out here from the ansatz for every equation.
* Two code paths: the exp network's field equals s q^{-k} exp(Phi_lin / (s q^{-k})) where
  Phi_lin is the same network's field under the linear map.
* The field jets' y-derivatives under exp match complex steps in y (first order) and central
  differences of those (second order).
"""
import numpy as np
import pytest

from oracle import problems as Pb
from paper_2509_14185_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

CASES = [(Pb.BURGERS, [1, 5, 1]), (Pb.CCF, [1, 5, 1]), (Pb.IPM, [2, 5, 2]), (Pb.BOUSSINESQ, [2, 5, 3])]


def envelope(eq, f, y, lam):
    """s_A q^{-k_A} of field f (parity class and exponent of each equation)."""
    u = 1.0 + np.sum(y * y, axis=0)
    q = u ** (-1.0 / (2.0 * (1.0 + lam)))
    odd = y[0] / np.sqrt(u)
    if eq == Pb.BURGERS:
        return odd * q ** (-lam)
    if eq == Pb.CCF:
        return (y[0] ** 2 / u) * q ** (-lam)
    if eq == Pb.IPM:
        return [q ** (-lam), odd * q ** (-(1.0 + 2.0 * lam))][f]
    return [odd * q, q ** (-(lam - 1.0)), odd * q ** (-(1.0 + 2.0 * lam))][f]


@pytest.mark.parametrize("eq,widths", CASES)
def test_constant_network_under_exp(eq, widths):
    w = I.small_case(eq, widths, 9, n_bnd=2, m=16)
    p = Pb.Problem(eq, widths, w.y, w.y_bnd, hilbert_m=16, output_map=1)
    theta = np.zeros(p.P)
    b = np.array([0.3, -0.7, 1.1])[: widths[-1]]
    theta[-widths[-1]:] = b
    lam = 0.45
    F = p.fields(theta, lam, w.y)
    for f in range(widths[-1]):
        np.testing.assert_allclose(F[f].v, envelope(eq, f, w.y, lam) * np.exp(b[f]), rtol=1e-13, atol=1e-300)


@pytest.mark.parametrize("eq,widths", CASES)
def test_exp_field_is_exp_of_linear_network(eq, widths):
    w = I.small_case(eq, widths, 11, n_bnd=2, m=16, seed=3)
    pl = Pb.Problem(eq, widths, w.y, w.y_bnd, hilbert_m=16)
    pe = Pb.Problem(eq, widths, w.y, w.y_bnd, hilbert_m=16, output_map=1)
    Fl, Fe = pl.fields(w.theta, w.lam, w.y), pe.fields(w.theta, w.lam, w.y)
    for f in range(widths[-1]):
        env = envelope(eq, f, w.y, w.lam)
        ok = np.abs(env) > 1e-6
        np.testing.assert_allclose(Fe[f].v[ok], env[ok] * np.exp(Fl[f].v[ok] / env[ok]), rtol=1e-12)


@pytest.mark.parametrize("eq,widths", [(Pb.CCF, [1, 6, 6, 1]), (Pb.BOUSSINESQ, [2, 6, 6, 3])])
def test_exp_field_jets_vs_complex_step(eq, widths):
    w = I.small_case(eq, widths, 6, m=16, seed=5)
    p = Pb.Problem(eq, widths, w.y, hilbert_m=16, output_map=1)
    ys = w.y
    F = p.fields(w.theta, w.lam, ys)
    d = p.d
    h = 1e-30
    e = 1e-5
    for i in range(d):
        yc = ys.astype(np.complex128)
        yc[i] += 1j * h
        dFi = [f.v.imag / h for f in p.fields(w.theta, w.lam, yc)]
        for f in range(widths[-1]):
            np.testing.assert_allclose(F[f].g[i], dFi[f], rtol=1e-12, atol=1e-14 * np.max(np.abs(dFi[f])))
        for j in range(d):   # second order: central difference in y_j of the complex-step d/dy_i
            out = []
            for s in (1.0, -1.0):
                yc2 = ys.astype(np.complex128)
                yc2[j] += s * e
                yc2[i] += 1j * h
                out.append([f.v.imag / h for f in p.fields(w.theta, w.lam, yc2)])
            for f in range(widths[-1]):
                fd = (out[0][f] - out[1][f]) / (2 * e)
                np.testing.assert_allclose(F[f].h[i][j], fd, rtol=1e-6, atol=1e-8 * np.max(np.abs(fd)))


# planted mistakes (on the CPU only): each pin above must fail when the oracle is wrong

def test_planted_wrong_second_derivative_breaks_jet_pin(monkeypatch):
    """exp with its second derivative dropped (the chain rule's f'' term set to 0)."""
    from oracle.jets import Jet

    def wrong(self):
        e = np.exp(self.v)
        return self.chain(e, e, 0.0 * e)
    monkeypatch.setattr(Jet, "exp", wrong)
    with pytest.raises(AssertionError):
        test_exp_field_jets_vs_complex_step(Pb.BOUSSINESQ, [2, 6, 6, 3])


def test_planted_exp_on_hidden_layer_breaks_two_path_pin(monkeypatch):
    """exp applied before the last linear layer instead of after it."""
    orig = Pb.Problem.mlp

    def wrong(self, theta, z, widths=None, fourier=None):
        if self.output_map != 1:
            return orig(self, theta, z, widths, fourier)
        h = z
        L = self.layers(theta, widths, fourier)
        for i, (W, b) in enumerate(L):
            a = h.matvec(W, b)
            h = a if i == len(L) - 1 else (a.tanh().exp() if i == len(L) - 2 else a.tanh())
        return h
    monkeypatch.setattr(Pb.Problem, "mlp", wrong)
    with pytest.raises(AssertionError):
        test_exp_field_is_exp_of_linear_network(Pb.IPM, [2, 5, 2])
