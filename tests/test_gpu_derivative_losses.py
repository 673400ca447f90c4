"""Derivative-loss rows on the GPU vs the oracle (Methods, "Training Loss": the d1 and d2 losses,
each with its own batch, point weights and coefficient).

For every equation a small fit with d1 and d2 batches (seeded subsets of the collocation points,
non-uniform point weights, c_d1 = 0.3, c_d2 = 0.05) goes through libgn and through the oracle
(`oracle/problems.py`: the residual operators on truncated Taylor series; for CCF the discrete
Hilbert velocity differentiated in the collocation point).  Compared: every row of r~ (the
derivative rows by themselves too), J~ per column, the adjoint gradient, one GN step, and the
captured graph step against the eager one.  Hidden widths above 32 make the lanes stride over
neurons; the point counts leave ragged warps.
"""
import numpy as np
import pytest

from oracle import gn as ogn
from paper_2509_14185_gb300 import inputs as I
from tests.gpu_cases import TOL, col_rel, dev, gpu_problem, host, oracle_problem, rel

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

CASES = {
    "burgers": (I.BURGERS, [1, 40, 40, 1], 60, 0, 16),
    "ccf": (I.CCF, [1, 40, 40, 1], 60, 0, 32),
    "ipm": (I.IPM, [2, 34, 34, 2], 48, 9, 16),
    "boussinesq": (I.BOUSSINESQ, [2, 33, 33, 3], 40, 7, 16),
}

_cache = {}


def case(name):
    if name not in _cache:
        eq, widths, n, nb, m = CASES[name]
        w = I.with_derivative_batches(I.small_case(eq, widths, n, n_bnd=nb, seed=13, m=m), 11, 9)
        p = oracle_problem(w)
        r = p.rows(w.theta, w.lam)
        J = ogn.jacobian(p, w.theta, w.lam)
        _cache[name] = (w, p, r, J)
    return _cache[name]


def drange(p):
    a = p.n * p.ne
    return a, a + p.n_d1 * p.ne * p.d + p.n_d2 * p.ne * p.d ** 2


@pytest.mark.parametrize("name", list(CASES))
def test_derivative_rows_and_jacobian(name):
    w, p, r_o, J_o = case(name)
    prob = gpu_problem(w)
    assert prob.n_rows == p.n_rows
    r, loss = prob.residual(dev(w.theta), w.lam)
    r = host(r)
    a, b = drange(p)
    assert b > a and np.max(np.abs(r_o[a:b])) > 0.0
    assert rel(r, r_o) <= TOL
    assert rel(r[a:b], r_o[a:b]) <= TOL                     # the derivative rows by themselves
    assert abs(loss - 0.5 * np.dot(r_o, r_o)) <= TOL * 0.5 * np.dot(r_o, r_o)
    J = host(prob.jacobian(dev(w.theta), w.lam))
    assert rel(J, J_o) <= TOL
    assert rel(J[a:b], J_o[a:b]) <= TOL
    assert col_rel(J, J_o, floor=1e-300) <= TOL
    # a row block cutting through the derivative rows equals the same rows of the whole Jacobian
    r0, nr = a - 3, (b - a) // 2 + 5
    Jb = host(prob.jacobian(dev(w.theta), w.lam, row0=r0, nrows=nr, ld=prob.P + 5))
    np.testing.assert_array_equal(Jb, J[r0:r0 + nr])
    prob.close()


@pytest.mark.parametrize("name", list(CASES))
def test_derivative_rows_gradient_and_step(name):
    w, p, r_o, J_o = case(name)
    prob = gpu_problem(w)
    g = host(prob.gradient(dev(w.theta), w.lam))
    assert rel(g, J_o.T @ r_o) <= TOL
    seed = np.random.default_rng(2).standard_normal(p.n_rows)
    gs = host(prob.gradient(dev(w.theta), w.lam, dev(seed)))
    assert rel(gs, J_o.T @ seed) <= TOL
    th_o, lam_o, gam_o, info_o = ogn.gn_step(p, w.theta, w.lam, w.gamma)
    theta = dev(w.theta)
    rc, lam, gam, info = prob.gn_step(theta, w.lam, w.gamma)
    assert rc == info_o["status"]
    assert abs(info["loss_before"] - info_o["loss_before"]) <= TOL * info_o["loss_before"]
    if rc == 0:
        assert info["alpha"] == info_o["alpha"]
        d_gpu = np.concatenate([w.theta - host(theta), [w.lam - lam]])
        d_o = np.concatenate([w.theta - th_o, [w.lam - lam_o]])
        cond = np.linalg.cond(info_o["G"] + info_o["gamma_used"] * np.eye(len(d_o)))
        assert rel(d_gpu, d_o) <= max(TOL, 1e-15 * cond)
        h_at_gpu = p.loss(host(theta), lam)
        assert abs(info["loss_after"] - h_at_gpu) <= TOL * h_at_gpu
    # the captured graph step equals the eager one bit for bit
    pg = gpu_problem(w)
    tg = dev(w.theta)
    rc_g, lam_g, gam_g, info_g = pg.gn_step_graph(tg, w.lam, w.gamma)
    assert rc_g == rc and lam_g == lam and gam_g == gam and info_g["loss_after"] == info["loss_after"]
    np.testing.assert_array_equal(host(tg), host(theta))
    prob.close()
    pg.close()


def test_derivative_rows_refuse_unsupported_networks():
    from paper_2509_14185_gb300 import gn
    w = I.with_derivative_batches(I.small_case(I.BURGERS, [1, 8, 8, 1], 20, seed=3), 4, 3)
    with pytest.raises(gn.GNError) as e:
        gpu_problem(w, output_map=1)
    assert e.value.code == gn.GN_ERR_UNSUPPORTED
