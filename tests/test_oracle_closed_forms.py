"""Closed-form pins: Burgers self-similar profiles and Hilbert transform pairs.

Burgers (the paper's worked example in the research-flowchart figure):
substituting y = -U - C U^(1 + 1/lambda) into R = -lambda U + ((1+lambda) y + U) U'
gives R = 0 identically; the profile is smooth iff 1 + 1/lambda is an odd
integer, i.e. lambda_n = 1/(2n + 2).  For lambda = 1/2, C = 1, U is the real
root of U^3 + U + y = 0 (Cardano); for lambda = 1/4, of U^5 + U + y = 0.

Hilbert: H[1/(1+s^2)](x) = x/(1+x^2), H[s/(1+s^2)](x) = -1/(1+x^2), and for the
CCF factorisation Theta = s g with g = s/(1+s^2): x H[g](x) = -x/(1+x^2).
Under s = tan(psi/2) these are trigonometric polynomials of degree 1, which
the M-point singularity-subtracted trapezoid rule integrates exactly for any
M >= 4, so the oracle's operator must reproduce them to rounding.
"""
import numpy as np
import pytest

from oracle import hilbert
from oracle import problems as Pb


def cardano(y):
    """Real root of U^3 + U + y = 0."""
    D = np.sqrt(y * y / 4 + 1.0 / 27)
    U = np.cbrt(-y / 2 + D) + np.cbrt(-y / 2 - D)
    for _ in range(3):   # Newton polish: Cardano's sum cancels for large |y|
        U = U - (U**3 + U + y) / (3 * U * U + 1)
    return U


def quintic_root(y):
    """Real root of U^5 + U + y = 0 by Newton from a safe start (monotone map)."""
    U = -np.cbrt(y) * (np.abs(y) > 1) - y * (np.abs(y) <= 1) / 2
    for _ in range(100):
        U = U - (U**5 + U + y) / (5 * U**4 + 1)
    return U


def test_burgers_cardano_profile_has_zero_residual():
    y = np.concatenate([-np.logspace(-3, 4, 200), np.logspace(-3, 4, 200)])
    U = cardano(y)
    assert np.max(np.abs(U**3 + U + y)) <= 1e-12 * np.max(np.abs(y))
    Uy = -1.0 / (1.0 + 3.0 * U * U)
    (R,) = Pb.residual_burgers(0.5, y, U, Uy)
    scale = np.abs(0.5 * U) + np.abs((1.5 * y + U) * Uy)
    assert np.max(np.abs(R) / scale) < 1e-13


def test_burgers_second_profile_lambda_quarter():
    y = np.concatenate([-np.logspace(-3, 3, 100), np.logspace(-3, 3, 100)])
    U = quintic_root(y)
    Uy = -1.0 / (1.0 + 5.0 * U**4)
    (R,) = Pb.residual_burgers(0.25, y, U, Uy)
    scale = np.abs(0.25 * U) + np.abs((1.25 * y + U) * Uy)
    assert np.max(np.abs(R) / scale) < 1e-13
    # a non-admissible lambda with the same profile leaves a clear residual
    (R2,) = Pb.residual_burgers(0.3, y, U, Uy)
    assert np.max(np.abs(R2) / scale) > 1e-3


@pytest.mark.parametrize("M", [8, 16, 64, 1024])
def test_hilbert_pairs_exact(M):
    x = np.concatenate([np.linspace(-5, 5, 37), np.logspace(-3, 4, 20)])
    h1 = hilbert.hilbert_decaying(x, lambda s: 1.0 / (1.0 + s * s), M)
    np.testing.assert_allclose(h1, x / (1 + x * x), rtol=0, atol=2e-14 * max(1, M / 64))
    h2 = hilbert.hilbert_decaying(x, lambda s: s / (1.0 + s * s), M)
    np.testing.assert_allclose(h2, -1.0 / (1 + x * x), rtol=0, atol=2e-14 * max(1, M / 64))


@pytest.mark.parametrize("M", [8, 128])
def test_ccf_velocity_factorised_pair(M):
    """U = x H[g] with g = s/(1+s^2), i.e. Theta = s^2/(1+s^2): U = -x/(1+x^2)."""
    x = np.concatenate([np.linspace(-4, 4, 33), np.logspace(-3, 4, 15)])
    _, s = hilbert.nodes(M)
    g = lambda v: v / (1.0 + v * v)
    U = hilbert.velocity(x, g(x), g(s), M)
    # U = x (C[G] - c0) cancels two O(1/2) terms: rounding scales with |x|
    err = np.abs(U + x / (1 + x * x))
    assert np.all(err <= 1e-15 * np.sqrt(M) * (1 + np.abs(x))), err.max()
