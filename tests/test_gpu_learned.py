"""The learned part: the MLP trained on the GPU by this project's kernels.

* GN training: damped Gauss-Newton steps (gn_step, FP64) fit the Burgers
  lambda = 1/2 profile; the trained network is compared with the method
  without a learned network, i.e. the same ansatz with NN == const (the best
  constant, found by a scan of gn_residual).  The exact profile is known in
  closed form (U^3 + U + y = 0, the paper's worked example in its research
  flowchart figure), so the gain is measured both in loss and in the error
  against the exact profile.
* Gradient training: the residual as a torch.autograd.Function (forward
  gn_residual, backward the adjoint kernel gn_gradient) drives torch's Adam;
  the same number of GN steps reaches a far lower loss (the paper's optimizer
  ablation, Methods "High-precision training" figure, in miniature).
"""
import numpy as np
import pytest
import torch

from paper_2509_14185_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def cardano(y):
    D = np.sqrt(y * y / 4 + 1.0 / 27)
    U = np.cbrt(-y / 2 + D) + np.cbrt(-y / 2 - D)
    for _ in range(3):
        U = U - (U ** 3 + U + y) / (3 * U * U + 1)
    return U


def burgers_problem(widths=(1, 24, 24, 1), seed=3):
    from paper_2509_14185_gb300 import gn
    y = np.concatenate([np.logspace(-2, 2, 150), np.linspace(0.02, 6.0, 106)]).reshape(1, -1)
    w = I.Workload(name="burgers_half", equation=I.BURGERS, widths=list(widths), y=y, y_bnd=np.zeros((1, 0)),
                   lam=0.5, theta=I.xavier_init(widths, seed), y_norm=(-2.0, 0.0), c_norm=1.0)
    return w, gn.GNProblem.from_workload(w)


def field_values(theta, lam, widths, ys):
    """U(y) of the Burgers ansatz on the CPU (only to compare with the closed form)."""
    from oracle import problems as Pb
    p = Pb.Problem(I.BURGERS, widths, ys.reshape(1, -1))
    return p.fields(theta, lam, ys.reshape(1, -1))[0].v


def const_theta(widths, c):
    th = np.zeros(I.param_count(widths))
    th[-1] = c          # output bias: NN == c
    return th


def test_gn_trained_network_beats_envelope_only_ansatz():
    w, prob = burgers_problem()
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    # the method without the learned part: NN == c, best c by a scan
    best = min((prob.gn_residual(dev(const_theta(w.widths, c)), 0.5)[1], c) for c in np.linspace(-3, 3, 241))
    loss_const, c_best = best
    # the learned part: GN training on the GPU
    theta = dev(w.theta)
    lam, gam = w.lam, 1e-4
    for _ in range(60):
        rc, lam, gam, info = prob.gn_step(theta, lam, gam)
        assert rc in (0, 1)
    loss_nn = prob.gn_residual(theta, lam)[1]
    assert loss_nn < 1e-3 * loss_const
    # max d0 residual on a validation grid covering the training range
    from paper_2509_14185_gb300 import gn
    grid = np.concatenate([np.logspace(-2, 2, 700), np.linspace(0.01, 6.0, 300)]).reshape(1, -1)
    val = gn.GNProblem(I.BURGERS, w.widths, grid, y_norm=w.y_norm, c_norm=w.c_norm)
    res_nn = val.gn_max_residual(theta, lam)
    res_c = val.gn_max_residual(dev(const_theta(w.widths, c_best)), 0.5)
    assert res_nn < 0.1 * res_c
    val.close()
    prob.close()


def test_gn_beats_adam_through_the_autograd_function():
    from paper_2509_14185_gb300.gn import residual_fn
    w, prob = burgers_problem(seed=4)
    theta0 = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    # Adam on h = |r~|^2 / 2, gradients from the adjoint kernel
    th = theta0.clone().requires_grad_(True)
    lam = torch.tensor(w.lam, dtype=torch.float64, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([th, lam], lr=3e-3)
    for _ in range(300):
        opt.zero_grad()
        r = residual_fn(th, lam, prob)
        loss = 0.5 * (r * r).sum()
        loss.backward()
        opt.step()
    loss_adam = prob.gn_residual(th.detach().contiguous(), float(lam))[1]
    # 30 GN steps from the same start
    theta = theta0.clone()
    l, gam = w.lam, 1e-4
    for _ in range(30):
        rc, l, gam, info = prob.gn_step(theta, l, gam)
    loss_gn = prob.gn_residual(theta, l)[1]
    assert loss_gn < 0.01 * loss_adam
    prob.close()
