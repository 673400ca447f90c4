"""Batched fits (gn_batch_*): stepping many uneven fits together on several streams
gives exactly the results of stepping each fit alone (every reduction in the
library has a fixed order, so the results are bitwise reproducible)."""
import numpy as np
import pytest
import torch

from paper_2509_14185_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def small_sweep(n=6):
    fits = []
    for f in range(n):
        w = 8 + 8 * (f % 3)
        depth = 2 + f % 2
        fits.append(I.small_case(I.CCF, [1] + [w] * depth + [1], 80 + 37 * f, seed=30 + f, m=32,
                                 lam=0.6 + 0.3 * f))
    return fits


@pytest.mark.parametrize("precision", [0, 2])
def test_batch_equals_sequential(precision):
    from paper_2509_14185_gb300 import gn
    fits = small_sweep()
    batch = gn.GNBatch(fits, n_streams=3, precision=precision, n_slices=6)
    thetas = [torch.tensor(w.theta, dtype=torch.float64, device="cuda") for w in fits]
    lams = [w.lam for w in fits]
    gams = [1e-4] * len(fits)
    for _ in range(3):
        lams, gams, infos, st = batch.gn_batch_step(thetas, lams, gams)
    # each fit alone
    for k, w in enumerate(fits):
        prob = gn.GNProblem.from_workload(w, precision=precision, n_slices=6)
        th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
        lam, gam = w.lam, 1e-4
        for _ in range(3):
            rc, lam, gam, info = prob.gn_step(th, lam, gam)
        assert np.array_equal(th.cpu().numpy(), thetas[k].cpu().numpy())
        assert lam == lams[k] and gam == gams[k]
        prob.close()
    batch.close()
