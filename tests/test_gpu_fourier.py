"""Fourier-feature networks (Methods, "Multi-stage Training", item 2) on the GPU against the
oracle: rows, Jacobian columns (B is not a parameter), the adjoint gradient and a GN step for
every equation; and the paper's second stage: a Fourier network learning the error of a
frozen stage-1 network."""
import copy

import numpy as np
import pytest

from oracle import gn as ogn
from oracle import lam as olam
from oracle import problems as Pb
from paper_2509_14185_gb300 import inputs as I
from tests.gpu_cases import CASES, TOL, col_rel, dev, host, rel, small

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def fourier_case(name, m=6, mf=5, h=10, sigma=3.0):
    w = copy.copy(small(name))
    d, nf = w.widths[0], w.widths[-1]
    w.widths = [d, m, 2 * mf, h, nf]
    B = sigma * I.normal(41, mf * m).reshape(mf, m)
    P = (d * m + m) + (2 * mf * h + h) + (h * nf + nf)
    w.theta = 0.5 * I.normal(43, P)
    return w, B


def oracle(w, B, stage1=None):
    return Pb.Problem(w.equation, w.widths, w.y, w.y_bnd if w.y_bnd.size else None, w.rho, y_norm=w.y_norm,
                      c_norm=w.c_norm, hilbert_m=w.hilbert_m, fourier=B, stage1=stage1)


def gpu(w, B, **kw):
    from paper_2509_14185_gb300 import gn
    return gn.GNProblem.from_workload(w, fourier_B=B, **kw)


@pytest.mark.parametrize("name", list(CASES))
def test_fourier_rows_jacobian_gradient_match_oracle(name):
    w, B = fourier_case(name)
    p = oracle(w, B)
    prob = gpu(w, B)
    assert prob.P == p.P
    th = dev(w.theta)
    r, _ = prob.residual(th, w.lam)
    r_o = p.rows(w.theta, w.lam)
    assert rel(host(r), r_o) <= TOL
    J = host(prob.jacobian(th, w.lam))
    J_o = ogn.jacobian(p, w.theta, w.lam)
    assert rel(J, J_o) <= TOL
    assert col_rel(J, J_o, floor=1e-300) <= TOL
    g = host(prob.gradient(th, w.lam))
    assert rel(g, J_o.T @ r_o) <= TOL
    prob.close()


@pytest.mark.parametrize("name", ["burgers", "ipm"])
def test_fourier_gn_step_matches_oracle(name):
    w, B = fourier_case(name)
    p = oracle(w, B)
    th_o, lam_o, gam_o, info_o = ogn.gn_step(p, w.theta, w.lam, 1e-4)
    prob = gpu(w, B)
    theta = dev(w.theta)
    rc, lam, gam, info = prob.gn_step(theta, w.lam, 1e-4)
    assert rc == info_o["status"]
    assert abs(info["loss_before"] - info_o["loss_before"]) <= TOL * info_o["loss_before"]
    if rc == 0:
        assert info["alpha"] == info_o["alpha"]
        d_gpu = np.concatenate([w.theta - host(theta), [w.lam - lam]])
        d_o = np.concatenate([w.theta - th_o, [w.lam - lam_o]])
        cond = np.linalg.cond(info_o["G"] + info_o["gamma_used"] * np.eye(len(d_o)))
        assert rel(d_gpu, d_o) <= max(TOL, 1e-15 * cond)
    prob.close()


@pytest.mark.parametrize("name", ["ccf", "boussinesq"])
def test_fourier_stage2_matches_oracle(name):
    """The paper's second stage: a Fourier network on Phi_1 + eps Phi_2 (rows / eps, lambda fixed)."""
    w1 = small(name)
    th1 = w1.theta + 0.2 * np.sin(np.arange(len(w1.theta)))
    w, B = fourier_case(name)
    eps = 1e-3
    p = oracle(w, B, stage1=(w1.widths, th1, eps))
    prob = gpu(w, B)
    prob.gn_set_stage1(w1.widths, dev(th1), w.lam, eps)
    th = dev(w.theta)
    r, _ = prob.residual(th, w.lam)
    assert rel(host(r), p.rows(w.theta, w.lam)) <= TOL
    J = host(prob.jacobian(th, w.lam))
    J_o = ogn.jacobian(p, w.theta, w.lam, cols=range(p.P))
    assert np.all(J[:, -1] == 0.0) and rel(J[:, :-1], J_o) <= TOL
    th_o, _, _, info_o = olam.frozen_gn_step(p, w.theta, w.lam, 1e-4)
    rc, lam, gam, info = prob.gn_step(th, w.lam, 1e-4)
    assert rc == info_o["status"] and lam == w.lam
    if rc == 0:
        cond = np.linalg.cond(info_o["G"] + info_o["gamma_used"] * np.eye(p.P))
        assert rel(w.theta - host(th), w.theta - th_o) <= max(TOL, 1e-15 * cond)
    prob.close()
