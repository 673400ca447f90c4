"""The exponential output map on the GPU against the oracle (Methods, "Solution Modeling":
exponential or exponential-adjacent last activation; linear is the default reading).

NN_A = exp(W_L h + b_L): the jet kernel maps the last layer's jets through exp (value, first
and second orders, and the q-direction third orders the lambda column needs) and pulls the
adjoints back through the same map.  Rows, every Jacobian column and the adjoint match the
oracle for each equation; one GN step; a stage-2 problem whose stage-1 network uses the map.
"""
import copy

import numpy as np
import pytest

from oracle import gn as ogn
from oracle import problems as Pb
from paper_2509_14185_gb300 import inputs as I
from tests.gpu_cases import CASES, TOL, col_rel, dev, gpu_problem, host, oracle_problem, rel, small

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def exp_case(name, seed=11):
    w = copy.copy(small(name, seed=seed))
    w.output_map = 1
    w.theta = 0.5 * w.theta   # keep exp of the outputs O(1)
    return w


@pytest.mark.parametrize("name", list(CASES))
def test_exp_output_rows_jacobian_adjoint(name):
    w = exp_case(name)
    p = oracle_problem(w)
    assert p.output_map == 1
    r_o = p.rows(w.theta, w.lam)
    J_o = ogn.jacobian(p, w.theta, w.lam)
    prob = gpu_problem(w)
    th = dev(w.theta)
    r, _ = prob.residual(th, w.lam)
    assert rel(host(r), r_o) <= TOL
    J = host(prob.jacobian(th, w.lam))
    assert rel(J, J_o) <= TOL
    assert col_rel(J, J_o, floor=1e-300) <= TOL
    g = host(prob.gradient(th, w.lam))
    assert rel(g, J_o.T @ r_o) <= TOL
    # the linear map on the same parameters gives other rows (the flag is live)
    wl = copy.copy(w)
    wl.output_map = 0
    pl = gpu_problem(wl)
    rl, _ = pl.residual(th, w.lam)
    assert rel(host(rl), r_o) > 1e-6
    prob.close()
    pl.close()


@pytest.mark.parametrize("name", ["burgers", "ipm"])
def test_exp_output_gn_step(name):
    w = exp_case(name, seed=5)
    p = oracle_problem(w)
    th_o, lam_o, gam_o, info_o = ogn.gn_step(p, w.theta, w.lam, w.gamma)
    prob = gpu_problem(w)
    theta = dev(w.theta)
    rc, lam, gam, info = prob.gn_step(theta, w.lam, w.gamma)
    assert rc == info_o["status"]
    assert abs(info["loss_before"] - info_o["loss_before"]) <= TOL * info_o["loss_before"]
    if rc == 0:
        assert info["alpha"] == info_o["alpha"]
        d_gpu = np.concatenate([w.theta - host(theta), [w.lam - lam]])
        A = info_o["G"] + info_o["gamma_used"] * np.eye(len(d_gpu))
        g_o = ogn.jacobian(p, w.theta, w.lam).T @ p.rows(w.theta, w.lam)
        delta = d_gpu / info["alpha"]
        be = np.max(np.abs(A @ delta - g_o)) / (np.max(np.abs(A)) * np.max(np.abs(delta)) + np.max(np.abs(g_o)))
        assert be <= 1e-12
    prob.close()


@pytest.mark.parametrize("name", ["ccf", "boussinesq"])
def test_exp_output_stage2(name):
    eps = 1e-3
    w1 = exp_case(name)
    d, nf = w1.widths[0], w1.widths[-1]
    th1 = w1.theta + 0.1 * np.sin(np.arange(len(w1.theta)))
    w2 = copy.copy(w1)
    w2.widths = [d, 12, 12, nf]
    w2.theta = 0.5 * I.xavier_init(w2.widths, 29)
    p2 = Pb.Problem(w2.equation, w2.widths, w2.y, w2.y_bnd if w2.y_bnd.size else None, w2.rho,
                    y_norm=w2.y_norm, c_norm=w2.c_norm, hilbert_m=w2.hilbert_m,
                    stage1=(w1.widths, th1, eps), output_map=1)
    prob = gpu_problem(w2)
    prob.gn_set_stage1(w1.widths, dev(th1), w2.lam, eps)
    th2 = dev(w2.theta)
    r, _ = prob.residual(th2, w2.lam)
    assert rel(host(r), p2.rows(w2.theta, w2.lam)) <= TOL
    J = host(prob.jacobian(th2, w2.lam))
    J_o = ogn.jacobian(p2, w2.theta, w2.lam, cols=range(p2.P))
    assert rel(J[:, :-1], J_o) <= TOL
    prob.close()
