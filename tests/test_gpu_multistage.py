"""Stage 2 of multi-stage training on the GPU (gn_set_stage1) against the oracle's stage-2
problem: rows, Jacobian columns and the damped GN step of Phi_1 + eps Phi_2 (rows / eps,
lambda fixed), every equation; the captured graph step equals the eager one."""
import copy

import numpy as np
import pytest

from oracle import gn as ogn
from oracle import lam as olam
from oracle import problems as Pb
from paper_2509_14185_gb300 import inputs as I
from tests.gpu_cases import CASES, TOL, col_rel, dev, gpu_problem, host, rel, small

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

EPS = 1e-3


def stage2_case(name):
    w1 = small(name)
    d, nf = w1.widths[0], w1.widths[-1]
    th1 = w1.theta + 0.2 * np.sin(np.arange(len(w1.theta)))
    w2 = copy.copy(w1)
    w2.widths = [d, 12, 12, nf]
    w2.theta = I.xavier_init(w2.widths, 29)
    p2 = Pb.Problem(w2.equation, w2.widths, w2.y, w2.y_bnd if w2.y_bnd.size else None, w2.rho,
                    y_norm=w2.y_norm, c_norm=w2.c_norm, hilbert_m=w2.hilbert_m,
                    stage1=(w1.widths, th1, EPS))
    return w1, th1, w2, p2


def gpu_stage2(w1, th1, w2, **kw):
    prob = gpu_problem(w2, **kw)
    prob.gn_set_stage1(w1.widths, dev(th1), w2.lam, EPS)
    return prob


@pytest.mark.parametrize("name", list(CASES))
def test_stage2_rows_and_jacobian_match_oracle(name):
    w1, th1, w2, p2 = stage2_case(name)
    prob = gpu_stage2(w1, th1, w2)
    th2 = dev(w2.theta)
    r, loss = prob.residual(th2, w2.lam)
    r_o = p2.rows(w2.theta, w2.lam)
    assert rel(host(r), r_o) <= TOL
    J = host(prob.jacobian(th2, w2.lam))
    J_o = ogn.jacobian(p2, w2.theta, w2.lam, cols=range(p2.P))
    assert np.all(J[:, -1] == 0.0)                 # lambda is held fixed in stage 2
    assert rel(J[:, :-1], J_o) <= TOL
    assert col_rel(J[:, :-1], J_o, floor=1e-300) <= TOL
    # max |R| of the composed field
    R = np.concatenate(p2.interior_residuals(w2.theta, w2.lam))
    assert abs(prob.gn_max_residual(th2, w2.lam) - np.max(np.abs(R))) <= 1e-10 * np.max(np.abs(R))
    prob.close()


@pytest.mark.parametrize("name", list(CASES))
def test_stage2_gn_step_matches_oracle(name):
    w1, th1, w2, p2 = stage2_case(name)
    th_o, lam_o, gam_o, info_o = olam.frozen_gn_step(p2, w2.theta, w2.lam, 1e-4)
    prob = gpu_stage2(w1, th1, w2)
    theta = dev(w2.theta)
    rc, lam, gam, info = prob.gn_step(theta, w2.lam, 1e-4)
    assert rc == info_o["status"] and lam == w2.lam
    assert abs(info["loss_before"] - info_o["loss_before"]) <= TOL * info_o["loss_before"]
    if rc == 0:
        assert info["alpha"] == info_o["alpha"]
        cond = np.linalg.cond(info_o["G"] + info_o["gamma_used"] * np.eye(p2.P))
        assert rel(w2.theta - host(theta), w2.theta - th_o) <= max(TOL, 1e-15 * cond)
    prob.close()


def test_stage2_graph_step_equals_eager():
    w1, th1, w2, p2 = stage2_case("ccf")
    pe = gpu_stage2(w1, th1, w2, precision=2, n_slices=6)
    pg = gpu_stage2(w1, th1, w2, precision=2, n_slices=6)
    te, tg = dev(w2.theta), dev(w2.theta)
    ge = gg = 1e-4
    for _ in range(3):
        rc_e, le, ge, _ = pe.gn_step(te, w2.lam, ge)
        rc_g, lg, gg, _ = pg.gn_step_graph(tg, w2.lam, gg)
        assert rc_e == rc_g and le == lg == w2.lam and ge == gg
    np.testing.assert_array_equal(host(tg), host(te))
    pe.close()
    pg.close()
