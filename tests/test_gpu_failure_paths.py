"""Failure paths of the C ABI, exercised without any GPU fault.

GN_ERR_NONFINITE: a NaN in theta or in a collocation point (host data) reaches the jet
kernel, which flags the non-finite residual row; gn_residual, gn_step and gn_step_graph
must return the code with theta and lambda untouched and without damping escalations.

GN_ERR_TIMEOUT: every mbarrier wait of the split-precision tensor-core kernels is bounded.
gn_test_bounded_waits shortens the bound to 20 ms and makes the kernels' producer issue no
copies, so no copy or MMA is ever in flight and the consumers' waits simply run out; the
kernel releases its tensor memory and returns, gn_gram / gn_damped_solve / gn_step return
GN_ERR_TIMEOUT, and after the hook is reset the same calls succeed on the same context with
the results of an undisturbed run.
"""
import ctypes

import numpy as np
import pytest
import torch

from tests.gpu_cases import dev, gpu_problem, host, small

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

GN_ERR_NONFINITE, GN_ERR_TIMEOUT = -4, -6


@pytest.mark.parametrize("name", ["ccf", "ipm"])
def test_nan_theta_returns_nonfinite(name):
    w = small(name)
    prob = gpu_problem(w, precision=2, n_slices=6)
    bad = w.theta.copy()
    bad[3] = np.nan
    rc, loss = prob.gn_residual(dev(bad), w.lam)
    assert rc == GN_ERR_NONFINITE and not np.isfinite(loss)
    for step in (prob.gn_step, prob.gn_step_graph):
        theta = dev(bad)
        before = host(theta).copy()
        rc, lam, gam, info = step(theta, w.lam, w.gamma)
        assert rc == GN_ERR_NONFINITE, (step.__name__, rc)
        assert info["chol_retries"] == 0
        np.testing.assert_array_equal(host(theta), before)
        assert lam == w.lam and gam == w.gamma
    # the handle stays usable: a finite theta steps normally afterwards
    theta = dev(w.theta)
    rc, lam, gam, info = prob.gn_step(theta, w.lam, w.gamma)
    assert rc in (0, 1) and np.isfinite(info["loss_before"])
    prob.close()


def test_nan_collocation_point_returns_nonfinite():
    w = small("burgers")
    y = w.y.copy()
    y[0, 7] = np.nan
    w.y = y
    prob = gpu_problem(w)
    rc, loss = prob.gn_residual(dev(w.theta), w.lam)
    assert rc == GN_ERR_NONFINITE
    theta = dev(w.theta)
    rc, lam, gam, info = prob.gn_step(theta, w.lam, w.gamma)
    assert rc == GN_ERR_NONFINITE
    np.testing.assert_array_equal(host(theta), w.theta)
    prob.close()


def test_bounded_waits_time_out_and_the_context_recovers():
    from paper_2509_14185_gb300 import gn
    L = gn.lib()
    w = small("ccf")
    prob = gpu_problem(w, precision=2, n_slices=6)
    Pp = prob.P + 1
    J = prob.jacobian(dev(w.theta), w.lam)
    r = torch.zeros(J.shape[0], dtype=torch.float64, device="cuda")
    G_ref = torch.zeros((Pp, Pp), dtype=torch.float64, device="cuda")
    g_ref = prob.new_vec(Pp)
    prob.gn_gram(J, J.shape[0], r, G_ref, g_ref, precision=1)   # also settles the split-K choice
    torch.cuda.synchronize()
    G = torch.full((Pp, Pp), 7.0, dtype=torch.float64, device="cuda")
    g = prob.new_vec(Pp)
    try:
        assert L.gn_test_bounded_waits(20_000_000, 1) == 0
        rc = L.gn_gram(prob.h, gn._ptr(J), J.stride(0), J.shape[0], gn._ptr(r), gn._ptr(G), gn._ptr(g), 1, 0)
        assert rc == GN_ERR_TIMEOUT
        delta = prob.new_vec(Pp)
        rc, gam, ret = prob.gn_damped_solve(G_ref, g_ref, 1e-6, delta)   # split factorisation's updates
        assert rc == GN_ERR_TIMEOUT
        theta = dev(w.theta)
        rc = L.gn_step(prob.h, gn._ptr(theta), ctypes.byref(ctypes.c_double(w.lam)),
                       ctypes.byref(ctypes.c_double(w.gamma)), None)
        assert rc == GN_ERR_TIMEOUT
        np.testing.assert_array_equal(host(theta), w.theta)
    finally:
        assert L.gn_test_bounded_waits(0, 0) == 0
    # same context, default bound, copies issued again: the Gram equals the undisturbed one
    torch.cuda.synchronize()
    prob.gn_gram(J, J.shape[0], r, G, g, precision=1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(np.tril(host(G)), np.tril(host(G_ref)))
    prob.close()
