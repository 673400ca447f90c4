"""Pins of the oracle's stage-2 problem (Methods, "Multi-stage Training"): the fields are
Phi_1 + eps Phi_2 with a frozen stage-1 network, and the rows are divided by eps.

* A stage-2 network whose output layer is zero gives exactly the stage-1 rows over eps
  (checked against a stage-1-only problem: an independent path).
* The paper's stage-2 equation, -eps D[Phi_1] Phi_2 + O(eps^2) = R_1: the composed
  residual R(Phi_1 + eps Phi_2) equals R_1 + eps D[Phi_1] Phi_2 up to O(eps^2), with the
  linear operator D taken independently by complex-step differentiation in eps."""
import warnings

import numpy as np
import pytest

from oracle import problems as Pb
from paper_2509_14185_gb300 import inputs as I

warnings.filterwarnings("ignore", category=RuntimeWarning)

CASES = {"burgers": (I.BURGERS, 1, 0), "ccf": (I.CCF, 1, 0), "ipm": (I.IPM, 2, 6), "boussinesq": (I.BOUSSINESQ, 3, 6)}


def setup(name, eps):
    eq, nf, nb = CASES[name]
    d = 2 if eq in (I.IPM, I.BOUSSINESQ) else 1
    w1 = [d, 10, 10, nf]
    w2 = [d, 8, 8, nf]
    w = I.small_case(eq, w1, 40, n_bnd=nb, seed=21, m=32)
    th1 = w.theta + 0.2 * np.sin(np.arange(len(w.theta)))
    th2 = I.xavier_init(w2, 22) + 0.1 * np.cos(np.arange(I.param_count(w2)))
    kw = dict(y_norm=w.y_norm, c_norm=w.c_norm, hilbert_m=w.hilbert_m)
    yb = w.y_bnd if w.y_bnd.size else None
    p1 = Pb.Problem(eq, w1, w.y, yb, **kw)
    p2 = Pb.Problem(eq, w2, w.y, yb, stage1=(w1, th1, eps), **kw)
    return w, p1, p2, th1, th2, w2


@pytest.mark.parametrize("name", list(CASES))
def test_zero_stage2_network_gives_stage1_rows_over_eps(name):
    eps = 3.7e-6
    w, p1, p2, th1, th2, w2 = setup(name, eps)
    nlast = w2[-2] * w2[-1] + w2[-1]
    th2z = th2.copy()
    th2z[-nlast:] = 0.0
    np.testing.assert_array_equal(p2.rows(th2z, w.lam), p1.rows(th1, w.lam) / eps)


@pytest.mark.parametrize("name", list(CASES))
def test_composed_residual_is_stage1_plus_eps_linearised_operator(name):
    w, p1, _, th1, th2, w2 = setup(name, 1.0)
    lam = w.lam
    R1 = np.concatenate(p1.interior_residuals(th1, lam))
    # D[Phi_1] Phi_2 by complex step in eps (exact to rounding for the analytic residual)
    pc = Pb.Problem(p1.eq, w2, p1.y, p1.y_bnd if p1.nb else None, y_norm=p1.y_norm, c_norm=p1.c_norm,
                    hilbert_m=p1.M, stage1=(p1.widths, th1, 1.0))
    h = 1e-30
    pc.stage1 = (p1.widths, th1, 1j * h)
    DPhi2 = np.concatenate(pc.interior_residuals(th2.astype(np.complex128), complex(lam))).imag / h
    errs = []
    for eps in (1e-3, 5e-4, 2.5e-4):
        pc.stage1 = (p1.widths, th1, eps)
        Re = np.concatenate(pc.interior_residuals(th2, lam))
        errs.append(np.max(np.abs(Re - R1 - eps * DPhi2)))
    scale = np.max(np.abs(DPhi2)) + np.max(np.abs(R1))
    # second order: halving eps divides the remainder by ~4 (or it is already at rounding)
    for a, b in zip(errs, errs[1:]):
        assert b <= 0.3 * a or b <= 1e-12 * scale, errs
    assert errs[0] <= 1e-3 * scale
