"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Each case runs the same seeded workload through libgn (reverse-mode jets on
the GPU) and through the oracle (complex-step forward mode on the CPU) and
compares r~, J~, g, G, the damped solve and one whole Gauss-Newton step.
"""
import numpy as np
import pytest
import torch

from tests.gpu_cases import (CASES, TOL, col_rel, dev, gpu_problem, host, oracle_problem, rel, small,
                             small_weighted)
from oracle import gn as ogn

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

_cache = {}


def oracle_rows_jac(name, weighted=False):
    key = (name, weighted)
    if key not in _cache:
        w = small_weighted(name) if weighted else small(name)
        p = oracle_problem(w)
        r = p.rows(w.theta, w.lam)
        J = ogn.jacobian(p, w.theta, w.lam)
        _cache[key] = (w, p, r, J)
    return _cache[key]


@pytest.mark.parametrize("name", list(CASES))
def test_residual_rows(name):
    w, p, r_o, _ = oracle_rows_jac(name)
    prob = gpu_problem(w)
    r, loss = prob.residual(dev(w.theta), w.lam)
    assert rel(host(r), r_o) <= TOL
    assert abs(loss - 0.5 * np.dot(r_o, r_o)) <= TOL * 0.5 * np.dot(r_o, r_o)


@pytest.mark.parametrize("name", list(CASES))
def test_jacobian_rows(name):
    w, p, r_o, J_o = oracle_rows_jac(name)
    prob = gpu_problem(w)
    J = host(prob.jacobian(dev(w.theta), w.lam))
    assert J.shape == J_o.shape
    assert rel(J, J_o) <= TOL
    assert col_rel(J, J_o, floor=1e-300) <= TOL
    # a row block in the middle (row-range API) equals the same rows of the full Jacobian
    r0, nr = p.n_rows // 3, p.n_rows // 4
    Jb = host(prob.jacobian(dev(w.theta), w.lam, row0=r0, nrows=nr, ld=prob.P + 9))
    np.testing.assert_array_equal(Jb, J[r0:r0 + nr])


@pytest.mark.parametrize("name", list(CASES))
def test_gradient_adjoint(name):
    w, p, r_o, J_o = oracle_rows_jac(name)
    prob = gpu_problem(w)
    g = host(prob.gradient(dev(w.theta), w.lam))
    assert rel(g, J_o.T @ r_o) <= TOL
    seed = np.random.default_rng(1).standard_normal(p.n_rows)
    gs = host(prob.gradient(dev(w.theta), w.lam, dev(seed)))
    assert rel(gs, J_o.T @ seed) <= TOL


@pytest.mark.parametrize("name", ["ccf", "boussinesq"])
def test_gram_fp64(name):
    w, p, r_o, J_o = oracle_rows_jac(name)
    prob = gpu_problem(w)
    Pp = prob.P + 1
    J = dev(J_o)
    G = torch.zeros((Pp, Pp), dtype=torch.float64, device="cuda")
    g = prob.new_vec(Pp)
    prob.gn_gram(J, J.shape[0], dev(r_o), G, g)
    Go = J_o.T @ J_o
    Gl = np.tril(host(G))
    assert rel(Gl, np.tril(Go)) <= TOL
    assert rel(host(g), J_o.T @ r_o) <= TOL
    # accumulate over two row blocks equals one pass
    h1 = J.shape[0] // 2
    G2 = torch.zeros_like(G)
    g2 = prob.new_vec(Pp)
    prob.gn_gram(J[:h1].contiguous(), h1, dev(r_o[:h1]), G2, g2)
    prob.gn_gram(J[h1:].contiguous(), J.shape[0] - h1, dev(r_o[h1:]), G2, g2, accumulate=True)
    assert rel(np.tril(host(G2)), np.tril(Go)) <= TOL


def test_damped_solve_and_not_spd():
    w, p, r_o, J_o = oracle_rows_jac("ccf")
    prob = gpu_problem(w)
    Go = J_o.T @ J_o
    go = J_o.T @ r_o
    delta = prob.new_vec(prob.P + 1)
    rc, gam, retries = prob.gn_damped_solve(dev(Go), dev(go), 1e-6, delta)
    assert rc == 0 and retries == 0 and gam == 1e-6
    d_o, _, _, ok = ogn.damped_solve(Go, go, 1e-6)
    A = Go + 1e-6 * np.eye(len(go))
    # normwise backward error of the GPU solve, and agreement with the oracle's solve
    res = np.max(np.abs(A @ host(delta) - go)) / (np.max(np.abs(A)) * np.max(np.abs(host(delta))))
    assert res <= 1e-13
    cond = np.linalg.cond(A)
    assert rel(host(delta), d_o) <= max(TOL, 1e-15 * cond)
    # an indefinite matrix: damping escalates 5 times, then GN_ERR_NOT_SPD
    neg = -np.eye(len(go)) * 1e9
    rc, gam, retries = prob.gn_damped_solve(dev(neg), dev(go), 1.0, delta)
    assert rc == -5 and retries == 5 and gam == pytest.approx(1e5)
    # escalation that succeeds: G = -0.5 I with gamma = 0.1 needs gamma = 1
    rc, gam, retries = prob.gn_damped_solve(dev(-0.5 * np.eye(len(go))), dev(go), 0.1, delta)
    assert rc == 0 and retries == 1 and gam == pytest.approx(1.0)
    np.testing.assert_allclose(host(delta), go / 0.5, rtol=1e-14)


@pytest.mark.parametrize("name", list(CASES))
def test_gn_step(name):
    w, p, r_o, J_o = oracle_rows_jac(name)
    th_o, lam_o, gam_o, info_o = ogn.gn_step(p, w.theta, w.lam, w.gamma)
    prob = gpu_problem(w)
    theta = dev(w.theta)
    rc, lam, gam, info = prob.gn_step(theta, w.lam, w.gamma)
    assert rc == info_o["status"]
    assert info["chol_retries"] == info_o["chol_retries"]
    assert abs(info["loss_before"] - info_o["loss_before"]) <= TOL * info_o["loss_before"]
    mr = p.max_abs_residual(w.theta, w.lam)      # max |R_k| at the starting point, unweighted
    assert abs(info["max_abs_res"] - mr) <= TOL * mr
    if rc == 0:
        assert info["alpha"] == info_o["alpha"]
        assert gam == pytest.approx(gam_o, rel=1e-15)
        # the step itself carries the conditioning of G + gamma I
        d_gpu = np.concatenate([w.theta - host(theta), [w.lam - lam]])
        d_o = np.concatenate([w.theta - th_o, [w.lam - lam_o]])
        cond = np.linalg.cond(info_o["G"] + info_o["gamma_used"] * np.eye(len(d_o)))
        assert rel(d_gpu, d_o) <= max(TOL, 1e-15 * cond)
        # the GPU's line-search loss is exact for the point it accepted ...
        h_at_gpu = p.loss(host(theta), lam)
        assert abs(info["loss_after"] - h_at_gpu) <= TOL * h_at_gpu
        # ... and that point differs from the oracle's by the step's conditioning
        assert abs(info["loss_after"] - info_o["loss_after"]) <= max(1e-10, 1e-15 * cond) * info_o["loss_before"]
    else:
        np.testing.assert_array_equal(host(theta), w.theta)
        assert lam == w.lam and gam == pytest.approx(gam_o, rel=1e-15)


@pytest.mark.parametrize("name", list(CASES))
def test_weighted_rows_jacobian_gradient_step(name):
    """Non-uniform point weights rho and non-unit wall and normalisation weights (the paper's
    d0 loss weights each point; its data loss a coefficient per constraint): r~, J~ per column,
    the adjoint gradient and one GN step against the oracle, whose weights are pinned to the
    paper's loss on the CPU."""
    w, p, r_o, J_o = oracle_rows_jac(name, weighted=True)
    assert w.rho is not None and w.c_bnd != 1.0 and w.c_norm_w != 1.0
    prob = gpu_problem(w)
    r, loss = prob.residual(dev(w.theta), w.lam)
    assert rel(host(r), r_o) <= TOL
    assert abs(loss - 0.5 * np.dot(r_o, r_o)) <= TOL * 0.5 * np.dot(r_o, r_o)
    J = host(prob.jacobian(dev(w.theta), w.lam))
    assert rel(J, J_o) <= TOL
    assert col_rel(J, J_o, floor=1e-300) <= TOL
    g = host(prob.gradient(dev(w.theta), w.lam))
    assert rel(g, J_o.T @ r_o) <= TOL
    th_o, lam_o, gam_o, info_o = ogn.gn_step(p, w.theta, w.lam, w.gamma)
    theta = dev(w.theta)
    rc, lam, gam, info = prob.gn_step(theta, w.lam, w.gamma)
    assert rc == info_o["status"]
    assert abs(info["loss_before"] - info_o["loss_before"]) <= TOL * info_o["loss_before"]
    mr = p.max_abs_residual(w.theta, w.lam)      # unweighted although rho is not 1
    assert abs(info["max_abs_res"] - mr) <= TOL * mr
    tg = dev(w.theta)
    rc_g, _, _, info_g = prob.gn_step_graph(tg, w.lam, w.gamma)
    assert rc_g == rc and info_g["max_abs_res"] == info["max_abs_res"]
    if rc == 0:
        assert info["alpha"] == info_o["alpha"]
        d_gpu = np.concatenate([w.theta - host(theta), [w.lam - lam]])
        d_o = np.concatenate([w.theta - th_o, [w.lam - lam_o]])
        cond = np.linalg.cond(info_o["G"] + info_o["gamma_used"] * np.eye(len(d_o)))
        assert rel(d_gpu, d_o) <= max(TOL, 1e-15 * cond)
    prob.close()


def test_autograd_function_backward():
    from paper_2509_14185_gb300.gn import residual_fn
    w, p, r_o, J_o = oracle_rows_jac("ipm")
    prob = gpu_problem(w)
    theta = dev(w.theta).requires_grad_(True)
    lam = torch.tensor(w.lam, dtype=torch.float64, device="cuda", requires_grad=True)
    r = residual_fn(theta, lam, prob)
    loss = 0.5 * (r * r).sum()
    loss.backward()
    g_o = J_o.T @ r_o
    assert rel(host(theta.grad), g_o[:-1]) <= TOL
    assert abs(lam.grad.item() - g_o[-1]) <= TOL * np.max(np.abs(g_o))


def test_empty_interior_and_single_layer():
    """Degenerate shapes: no interior points (only the normalisation row) and a
    network with no hidden layer."""
    from paper_2509_14185_gb300 import inputs as I
    w = I.small_case(I.BURGERS, [1, 1], 0, seed=3)
    p = oracle_problem(w)
    prob = gpu_problem(w)
    assert prob.n_rows == 1 and prob.P == 2
    r, _ = prob.residual(dev(w.theta), w.lam)
    assert rel(host(r), p.rows(w.theta, w.lam)) <= TOL
    J = host(prob.jacobian(dev(w.theta), w.lam))
    assert rel(J, ogn.jacobian(p, w.theta, w.lam)) <= TOL
    w2 = I.small_case(I.IPM, [2, 2], 33, n_bnd=5, seed=4)
    p2 = oracle_problem(w2)
    prob2 = gpu_problem(w2)
    J2 = host(prob2.jacobian(dev(w2.theta), w2.lam))
    assert rel(J2, ogn.jacobian(p2, w2.theta, w2.lam)) <= TOL


@pytest.mark.parametrize("name", ["burgers", "ccf", "ipm"])
@pytest.mark.parametrize("precision", [0, 2])
def test_row_blocks(name, precision):
    """gn_problem.row_block: the Jacobian streamed in blocks of 97 rows (several blocks and a
    ragged last one), the Gram accumulated over them.  Steps agree with the oracle's (the
    accumulation order differs from one pass, so within the step's conditioning), and the
    captured graph step equals the eager one bit for bit."""
    w, p, r_o, J_o = oracle_rows_jac(name)
    th_o, lam_o, gam_o, info_o = ogn.gn_step(p, w.theta, w.lam, w.gamma)
    prob = gpu_problem(w, precision=precision, n_slices=6, row_block=97)
    pg = gpu_problem(w, precision=precision, n_slices=6, row_block=97)
    theta, tg = dev(w.theta), dev(w.theta)
    rc, lam, gam, info = prob.gn_step(theta, w.lam, w.gamma)
    rc_g, lam_g, gam_g, info_g = pg.gn_step_graph(tg, w.lam, w.gamma)
    assert rc == rc_g and lam == lam_g and gam == gam_g and info["loss_after"] == info_g["loss_after"]
    np.testing.assert_array_equal(host(tg), host(theta))
    if precision == 0:
        assert rc == info_o["status"]
        assert abs(info["loss_before"] - info_o["loss_before"]) <= TOL * info_o["loss_before"]
        if rc == 0:
            d_gpu = np.concatenate([w.theta - host(theta), [w.lam - lam]])
            d_o = np.concatenate([w.theta - th_o, [w.lam - lam_o]])
            cond = np.linalg.cond(info_o["G"] + info_o["gamma_used"] * np.eye(len(d_o)))
            assert rel(d_gpu, d_o) <= max(TOL, 1e-13 * cond)
    prob.close()
    pg.close()
