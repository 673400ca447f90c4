"""Pins of the oracle's Fourier-feature network (Methods, "Multi-stage Training", item 2:
a fixed map [cos(B x), sin(B x)] after the linear input layer):
* a network whose Fourier layer feeds the output layer directly has a closed form,
  NN(z) = w1 cos(b (W0 z + b0)) + w2 sin(b (W0 z + b0)) + c, checked with its first and
  second derivatives;
* the field jets of a deep Fourier network in 2D agree with complex-step derivatives in y;
* B is not a parameter: P counts the trainable layers only."""
import warnings

import numpy as np
import pytest

from oracle import problems as Pb
from oracle.jets import Jet
from paper_2509_14185_gb300 import inputs as I

warnings.filterwarnings("ignore", category=RuntimeWarning)


def test_shallow_fourier_network_closed_form():
    widths = [1, 1, 2, 1]
    bmat = np.array([[1.7]])
    y = np.array([[0.3, 1.0, 4.0]])
    p = Pb.Problem(I.BURGERS, widths, y, fourier=bmat)
    W0, b0, w1, w2, c = 0.8, -0.25, 0.6, -1.3, 0.05
    theta = np.array([W0, b0, w1, w2, c])
    assert p.P == 5
    z = np.array([0.2, 0.55, 0.9])
    zj = Jet(z.reshape(1, -1), [np.ones((1, 3))], [[np.zeros((1, 3))]])
    out = p.mlp(theta, zj, fourier=bmat)
    arg = 1.7 * (W0 * z + b0)
    k = 1.7 * W0
    v = w1 * np.cos(arg) + w2 * np.sin(arg) + c
    d1 = k * (-w1 * np.sin(arg) + w2 * np.cos(arg))
    d2 = -k * k * (w1 * np.cos(arg) + w2 * np.sin(arg))
    np.testing.assert_allclose(out.v[0], v, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(out.g[0][0], d1, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(out.h[0][0][0], d2, rtol=1e-13, atol=1e-15)


def test_fourier_field_jets_match_complex_step_in_y():
    widths = [2, 6, 8, 10, 3]
    rng = np.random.default_rng(4)
    bmat = rng.normal(0.0, 3.0, size=(4, 6))
    pts = np.array([[0.3, 2.0, 0.01], [0.7, 0.1, 5.0]])
    p = Pb.Problem(I.BOUSSINESQ, widths, pts, fourier=bmat)
    assert p.P == (2 * 6 + 6) + (8 * 10 + 10) + (10 * 3 + 3)
    theta = 0.4 * rng.standard_normal(p.P)
    lam = 1.7
    F = p.fields(theta, lam, pts)
    h = 1e-30
    for k in range(2):
        yc = pts.astype(np.complex128)
        yc[k] += 1j * h
        Fc = p.fields(theta.astype(np.complex128), complex(lam), yc)
        for f in range(3):
            np.testing.assert_allclose(F[f].g[k], Fc[f].v.imag / h, rtol=1e-12, atol=1e-14)
            # second derivatives: complex step of the first-derivative jet
            for j in range(2):
                np.testing.assert_allclose(F[f].h[j][k], Fc[f].g[j].imag / h, rtol=1e-11, atol=1e-12)
