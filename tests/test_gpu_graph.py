"""Graph-captured steps (gn_step_graph, gn_batch_capture_graph / gn_batch_graph_step).

The captured step moves gn_step's host decisions (factorisation check, Armijo
backtracking, Levenberg-Marquardt update) into device kernels around the same
launch sequence, so it must reproduce gn_step exactly: same kernels, same
reduction orders, and decisions on the same FP64 values.  One case is also
checked against the CPU oracle directly.
"""
import numpy as np
import pytest
import torch

from oracle import gn as ogn
from tests.gpu_cases import CASES, TOL, dev, gpu_problem, host, oracle_problem, rel, small
from tests.test_gpu_batch import small_sweep

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def run(prob, theta, lam, gam, steps, graph):
    out = []
    for _ in range(steps):
        f = prob.gn_step_graph if graph else prob.gn_step
        rc, lam, gam, info = f(theta, lam, gam)
        out.append((rc, lam, gam, info))
    return out


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("name", list(CASES))
def test_graph_step_equals_eager(name, precision):
    w = small(name)
    pe = gpu_problem(w, precision=precision, n_slices=6)
    pg = gpu_problem(w, precision=precision, n_slices=6)
    te, tg = dev(w.theta), dev(w.theta)
    gam0 = 1e-4
    eager = run(pe, te, w.lam, gam0, 4, graph=False)
    graph = run(pg, tg, w.lam, gam0, 4, graph=True)
    for (rc_e, lam_e, gam_e, ie), (rc_g, lam_g, gam_g, ig) in zip(eager, graph):
        assert rc_g == rc_e
        assert ig["n_trials"] == ie["n_trials"] and ig["chol_retries"] == ie["chol_retries"]
        assert lam_g == lam_e and gam_g == gam_e
        assert ig["alpha"] == ie["alpha"] and ig["gamma_used"] == ie["gamma_used"]
        assert ig["loss_before"] == ie["loss_before"] and ig["loss_after"] == ie["loss_after"]
        assert ig["rho"] == pytest.approx(ie["rho"], rel=1e-12, abs=1e-300)
    np.testing.assert_array_equal(host(tg), host(te))
    # a new theta buffer recaptures; a second handle stepping the same theta gives the same
    t2 = dev(host(te))
    rc1, lam1, gam1, _ = pg.gn_step_graph(t2, eager[-1][1], eager[-1][2])
    rc2, lam2, gam2, _ = pe.gn_step(te, eager[-1][1], eager[-1][2])
    assert rc1 == rc2 and lam1 == lam2 and gam1 == gam2
    np.testing.assert_array_equal(host(t2), host(te))
    pe.close()
    pg.close()


def test_graph_step_matches_oracle():
    w = small("ccf")
    p = oracle_problem(w)
    th_o, lam_o, gam_o, info_o = ogn.gn_step(p, w.theta, w.lam, w.gamma)
    prob = gpu_problem(w)
    theta = dev(w.theta)
    rc, lam, gam, info = prob.gn_step_graph(theta, w.lam, w.gamma)
    assert rc == info_o["status"] == 0
    assert info["alpha"] == info_o["alpha"]
    assert gam == pytest.approx(gam_o, rel=1e-15)
    assert abs(info["loss_before"] - info_o["loss_before"]) <= TOL * info_o["loss_before"]
    d_gpu = np.concatenate([w.theta - host(theta), [w.lam - lam]])
    d_o = np.concatenate([w.theta - th_o, [w.lam - lam_o]])
    cond = np.linalg.cond(info_o["G"] + info_o["gamma_used"] * np.eye(len(d_o)))
    assert rel(d_gpu, d_o) <= max(TOL, 1e-15 * cond)
    # the phase marks inside the graph time the Jacobian, the Gram and the solve
    ph = info["ms_phase"]
    assert ph[0] > 0 and ph[1] > 0 and ph[3] > 0 and ph[5] > 0
    assert ph[0] + ph[1] + ph[3] + ph[4] + ph[5] <= ph[6] * 1.001
    prob.close()


def test_graph_step_not_spd_retries():
    """A negative damping makes every factorisation fail: the solve graph is replayed with
    damping x10 five times, then GN_ERR_NOT_SPD with theta and lambda untouched (as gn_step)."""
    w = small("burgers")
    pe, pg = gpu_problem(w), gpu_problem(w)
    te, tg = dev(w.theta), dev(w.theta)
    rc_e, lam_e, gam_e, ie = pe.gn_step(te, w.lam, -1e3)
    rc_g, lam_g, gam_g, ig = pg.gn_step_graph(tg, w.lam, -1e3)
    assert rc_e == rc_g == -5
    assert ig["chol_retries"] == ie["chol_retries"] == 5
    assert ig["gamma_used"] == ie["gamma_used"]
    assert lam_g == w.lam and gam_g == gam_e
    np.testing.assert_array_equal(host(tg), w.theta)
    # the handle keeps working after the failure
    rc, lam, gam, info = pg.gn_step_graph(tg, w.lam, 1e-4)
    rc2, lam2, gam2, info2 = pe.gn_step(te, w.lam, 1e-4)
    assert rc == rc2 and lam == lam2 and gam == gam2
    np.testing.assert_array_equal(host(tg), host(te))
    pe.close()
    pg.close()


@pytest.mark.parametrize("precision", [0, 2])
def test_batch_graph_equals_eager_batch(precision):
    from paper_2509_14185_gb300 import gn
    fits = small_sweep()
    be = gn.GNBatch(fits, n_streams=3, precision=precision, n_slices=6)
    bg = gn.GNBatch(fits, n_streams=3, precision=precision, n_slices=6)
    te = [torch.tensor(w.theta, dtype=torch.float64, device="cuda") for w in fits]
    tg = [torch.tensor(w.theta, dtype=torch.float64, device="cuda") for w in fits]
    le, lg = [w.lam for w in fits], [w.lam for w in fits]
    ge, gg = [1e-4] * len(fits), [1e-4] * len(fits)
    bg.gn_batch_capture_graph(tg)
    for _ in range(3):
        le, ge, ie, se = be.gn_batch_step(te, le, ge)
        lg, gg, ig, sg = bg.gn_batch_graph_step(lg, gg)
        assert sg == se
        assert [i["n_trials"] for i in ig] == [i["n_trials"] for i in ie]
    assert lg == le and gg == ge
    for k in range(len(fits)):
        np.testing.assert_array_equal(tg[k].cpu().numpy(), te[k].cpu().numpy())
    be.close()
    bg.close()
