"""The paper's own optimiser (gn_step_ema: EMA of rank-1 curvature estimates with
closed-form learning rate and momentum) against the oracle's ema_step, step by step
from the same seeded sign vectors; and a head-to-head with the exact-G step on the
same kernels."""
import numpy as np
import pytest
import torch

from oracle import gn as ogn
from paper_2509_14185_gb300 import inputs as I
from tests.gpu_cases import dev, gpu_problem, host, oracle_problem, small

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.mark.parametrize("name,precision", [("ccf", 0), ("burgers", 0), ("ipm", 0), ("ccf", 2)])
def test_ema_steps_match_oracle(name, precision):
    w = small(name)
    p = oracle_problem(w)
    prob = gpu_problem(w, precision=precision, n_slices=6)
    Pp, R = p.P + 1, p.n_rows
    theta_o, lam_o, gam_o = w.theta.copy(), w.lam, 1e-3
    G_o, v_o = np.zeros((Pp, Pp)), np.zeros(Pp)
    theta = dev(w.theta)
    lam, gam = w.lam, 1e-3
    G = torch.zeros((Pp, Pp), dtype=torch.float64, device="cuda")
    v = torch.zeros(Pp, dtype=torch.float64, device="cuda")
    beta = 0.9
    prev_tol = 0.0
    for k in range(3):
        s = I.signs(77, R, R * k)
        theta_o, lam_o, gam_o, G_o, v_o, info_o = ogn.ema_step(p, theta_o, lam_o, gam_o, G_o, v_o, s, beta, k == 0)
        rc, lam, gam, info = prob.gn_step_ema(theta, lam, gam, G, v, dev(s), beta, k == 0)
        assert rc == info_o["status"] == 0
        # the step goes through the damped solve: its error scales with cond(G_ema + gamma I)
        # (backward error ~1e-15 on the FP64 path, ~2e-13 for the split factor; x10 margin)
        cond = np.linalg.cond(G_o + info_o["gamma_used"] * np.eye(Pp))
        tol = max(1e-10, (1e-14 if precision == 0 else 2e-12) * cond)
        # the first average is u u^T of the sampled u = J~^T v alone: as tight as J~; later ones
        # also carry the previous step's difference in theta
        gtol = 1e-11 if k == 0 else max(1e-11, 10 * prev_tol)
        assert np.max(np.abs(host(G) - G_o)) <= gtol * np.max(np.abs(G_o))
        prev_tol = tol
        assert abs(info["alpha"] - info_o["alpha"]) <= tol * max(1.0, abs(info_o["alpha"]))
        assert abs(info["momentum"] - info_o["mu"]) <= tol * max(1.0, abs(info_o["mu"]))
        x = np.concatenate([host(theta), [lam]])
        xo = np.concatenate([theta_o, [lam_o]])
        assert np.max(np.abs(x - xo)) <= tol * np.max(np.abs(xo))
        assert np.max(np.abs(host(v) - v_o)) <= tol * np.max(np.abs(v_o))
        # (an early rank-1 average can overshoot, so the new loss may exceed the old one: compare
        # relative to the larger of the two, with the loss's own sensitivity to theta as margin)
        assert abs(info["loss_after"] - info_o["loss_after"]) <= 100 * tol * max(info_o["loss_before"],
                                                                                  info_o["loss_after"])
        assert gam == pytest.approx(gam_o, rel=1e-12) or abs(info["rho"] - info_o["rho"]) < 1e-6
    prob.close()


def test_ema_refuses_bad_beta():
    from paper_2509_14185_gb300 import gn
    w = small("ccf")
    prob = gpu_problem(w)
    Pp = prob.P + 1
    G = torch.zeros((Pp, Pp), dtype=torch.float64, device="cuda")
    v = torch.zeros(Pp, dtype=torch.float64, device="cuda")
    with pytest.raises(gn.GNError):
        prob.gn_step_ema(dev(w.theta), w.lam, 1e-3, G, v, dev(np.ones(prob.n_rows)), 1.0, True)
    prob.close()
