"""Decay rows of the data loss on the GPU against the oracle.

The normalised field Phi_A0 must vanish at far points Y_inf (Methods, "Training Loss",
second data-loss term); each point is one row sqrt(2 c_inf) Phi_A0(y) between the wall rows
and the normalisation row.  Rows, Jacobian columns (the lambda column included) and the
adjoint match the oracle for every equation; the decay rows also compose with stage 2 of
multi-stage training; a SPLIT_ALL graph step with decay rows equals the eager step.
"""
import copy

import numpy as np
import pytest

from oracle import gn as ogn
from oracle import problems as Pb
from paper_2509_14185_gb300 import inputs as I
from tests.gpu_cases import CASES, TOL, col_rel, dev, gpu_problem, host, oracle_problem, rel, small

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

N_INF = 37   # more than one warp's worth and not a multiple of the block


def with_decay(name, seed=11):
    w = copy.copy(small(name, seed=seed))
    rng = np.random.default_rng(seed + 100)
    r = 10.0 ** rng.uniform(0.5, 2.5, N_INF)
    if w.d == 1:
        w.y_inf = (r * rng.choice([-1.0, 1.0], N_INF)).reshape(1, N_INF)
    else:
        a = rng.uniform(0.0, np.pi / 2, N_INF)
        w.y_inf = np.stack([r * np.cos(a), r * np.sin(a)])
    w.c_inf = 0.3
    return w


@pytest.mark.parametrize("name", list(CASES))
def test_decay_rows_match_oracle(name):
    w = with_decay(name)
    p = oracle_problem(w)
    assert p.ninf == N_INF
    r_o = p.rows(w.theta, w.lam)
    J_o = ogn.jacobian(p, w.theta, w.lam)
    prob = gpu_problem(w)
    assert prob.n_rows == p.n_rows
    th = dev(w.theta)
    r, loss = prob.residual(th, w.lam)
    assert rel(host(r), r_o) <= TOL
    lo = p.n * p.ne + p.nb
    assert rel(host(r)[lo:lo + N_INF], r_o[lo:lo + N_INF]) <= TOL
    J = host(prob.jacobian(th, w.lam))
    assert rel(J, J_o) <= TOL
    assert col_rel(J, J_o, floor=1e-300) <= TOL
    assert rel(J[lo:lo + N_INF], J_o[lo:lo + N_INF]) <= TOL
    g = host(prob.gradient(th, w.lam))
    assert rel(g, J_o.T @ r_o) <= TOL
    prob.close()


@pytest.mark.parametrize("name", ["burgers", "ipm"])
def test_decay_rows_gn_step_matches_oracle(name):
    """Far decay points make G + gamma I ill-conditioned (cond ~1e9 for Burgers).  The two
    sides' G agree to the Jacobian's parity level (~1e-14 relative), so their steps may
    differ by cond times that; what is well-posed is that the GPU step solves the oracle's
    damped normal equations to a backward error of rounding size."""
    w = with_decay(name, seed=5)
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
        d_o = np.concatenate([w.theta - th_o, [w.lam - lam_o]])
        A = info_o["G"] + info_o["gamma_used"] * np.eye(len(d_o))
        g_o = ogn.jacobian(p, w.theta, w.lam).T @ p.rows(w.theta, w.lam)
        delta = d_gpu / info["alpha"]
        be = np.max(np.abs(A @ delta - g_o)) / (np.max(np.abs(A)) * np.max(np.abs(delta)) + np.max(np.abs(g_o)))
        assert be <= 1e-12
        assert rel(d_gpu, d_o) <= max(TOL, 1e-13 * np.linalg.cond(A))
    prob.close()


@pytest.mark.parametrize("name", ["ccf", "boussinesq"])
def test_decay_rows_in_stage2(name):
    eps = 1e-3
    w1 = small(name)
    d, nf = w1.widths[0], w1.widths[-1]
    th1 = w1.theta + 0.2 * np.sin(np.arange(len(w1.theta)))
    w2 = with_decay(name)
    w2.widths = [d, 12, 12, nf]
    w2.theta = I.xavier_init(w2.widths, 29)
    p2 = Pb.Problem(w2.equation, w2.widths, w2.y, w2.y_bnd if w2.y_bnd.size else None, w2.rho,
                    y_norm=w2.y_norm, c_norm=w2.c_norm, hilbert_m=w2.hilbert_m,
                    stage1=(w1.widths, th1, eps), y_inf=w2.y_inf, c_inf=w2.c_inf)
    prob = gpu_problem(w2)
    prob.gn_set_stage1(w1.widths, dev(th1), w2.lam, eps)
    th2 = dev(w2.theta)
    r, _ = prob.residual(th2, w2.lam)
    assert rel(host(r), p2.rows(w2.theta, w2.lam)) <= TOL
    J = host(prob.jacobian(th2, w2.lam))
    J_o = ogn.jacobian(p2, w2.theta, w2.lam, cols=range(p2.P))
    assert rel(J[:, :-1], J_o) <= TOL
    prob.close()


def test_decay_rows_graph_step_equals_eager():
    w = with_decay("ipm", seed=3)
    pe = gpu_problem(w, precision=2, n_slices=6)
    pg = gpu_problem(w, precision=2, n_slices=6)
    te, tg = dev(w.theta), dev(w.theta)
    le = lg = w.lam
    ge = gg = 1e-4
    for _ in range(3):
        rc_e, le, ge, ie = pe.gn_step(te, le, ge)
        rc_g, lg, gg, ig = pg.gn_step_graph(tg, lg, gg)
        assert rc_e == rc_g and ie["n_trials"] == ig["n_trials"] and ie["loss_after"] == ig["loss_after"]
    assert le == lg and ge == gg
    np.testing.assert_array_equal(host(tg), host(te))
    pe.close()
    pg.close()


@pytest.mark.parametrize("name,field,deriv", [("burgers", 0, 1), ("ipm", 1, 0), ("ipm", 1, 1),
                                              ("boussinesq", 2, 0), ("boussinesq", 1, 1)])
def test_normalisation_on_another_field_or_derivative(name, field, deriv):
    """The normalisation row on any field, value or d/dy1 (Methods, "Training Loss"); the decay
    rows follow that field: rows, Jacobian columns and the adjoint vs the oracle."""
    w = with_decay(name, seed=7)
    w.norm_field, w.norm_deriv = field, deriv
    p = oracle_problem(w)
    assert p.norm_field == field and p.norm_deriv == deriv
    r_o = p.rows(w.theta, w.lam)
    J_o = ogn.jacobian(p, w.theta, w.lam)
    prob = gpu_problem(w)
    th = dev(w.theta)
    r, _ = prob.residual(th, w.lam)
    assert rel(host(r), r_o) <= TOL
    assert abs(host(r)[-1] - r_o[-1]) <= TOL * max(abs(r_o[-1]), np.max(np.abs(r_o)))
    J = host(prob.jacobian(th, w.lam))
    assert rel(J, J_o) <= TOL
    assert rel(J[-1], J_o[-1]) <= TOL
    g = host(prob.gradient(th, w.lam))
    assert rel(g, J_o.T @ r_o) <= TOL
    prob.close()


@pytest.mark.parametrize("name,sign", [("burgers", 1), ("ipm", -1), ("boussinesq", 1), ("ccf", -1)])
def test_relu_bound_rows_match_oracle(name, sign):
    """Bound rows relu(s (Phi_A0 - b)) (Methods, "Training Loss"): the bound sits between two
    points' field values (no point at the kink), so about half the rows are active; rows,
    Jacobian columns (zero rows where inactive) and the adjoint vs the oracle."""
    w = with_decay(name, seed=13)
    yb = (w.y_inf * 0.01)[:, :29]
    vals = np.sort(oracle_problem(w).fields(w.theta, w.lam, yb)[0].v)
    w.y_relu, w.c_relu, w.relu_bound, w.relu_sign = yb, 0.9, float(0.5 * (vals[14] + vals[15])), sign
    p = oracle_problem(w)
    assert p.nrelu == 29
    r_o = p.rows(w.theta, w.lam)
    J_o = ogn.jacobian(p, w.theta, w.lam)
    lo = p.n * p.ne + p.nb + p.ninf
    active = r_o[lo:lo + 29] != 0.0
    assert 10 <= active.sum() <= 19
    prob = gpu_problem(w)
    th = dev(w.theta)
    r, _ = prob.residual(th, w.lam)
    r = host(r)
    assert rel(r, r_o) <= TOL
    np.testing.assert_array_equal(r[lo:lo + 29] != 0.0, active)
    J = host(prob.jacobian(th, w.lam))
    assert rel(J, J_o) <= TOL
    assert np.all(J[lo:lo + 29][~active] == 0.0)
    g = host(prob.gradient(th, w.lam))
    assert rel(g, J_o.T @ r_o) <= TOL
    prob.close()
