"""Funnel inference end to end on the GPU (Methods, "Identifying Admissible lambda Values",
item 3) on the paper's worked example, whose admissible rates are known in closed form:
Burgers has smooth self-similar profiles only for lambda = 1/(2n + 2), so fits started at
lambda 0.45 .. 0.55, each trained at fixed lambda and moved by the secant on the signed
residual near the origin, must converge to lambda = 1/2."""
import statistics

import pytest
import torch

from paper_2509_14185_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def test_funnel_inference_finds_the_admissible_burgers_lambda():
    from paper_2509_14185_gb300 import gn
    seeds = [0.45, 0.48, 0.52, 0.55]
    fits = []
    for f, lam in enumerate(seeds):
        w = I.burgers_half_1d(seed=106 + f)
        w.lam = lam
        fits.append(w)
    batch = gn.GNBatch(fits, n_streams=4, precision=gn.GN_PREC_SPLIT_ALL, n_slices=6)
    batch.gn_set_lambda_trainable(False)
    thetas = [torch.tensor(w.theta, dtype=torch.float64, device="cuda") for w in fits]
    batch.gn_batch_capture_graph(thetas)
    lams = list(seeds)
    gams = [w.gamma for w in fits]
    hist_l = [[l] for l in lams]
    hist_r = [[] for _ in fits]
    for _ in range(1200):                      # relax at the seed lambdas
        lams2, gams, infos, st = batch.gn_batch_graph_step(lams, gams)
        assert lams2 == lams
    for it in range(7):
        for _ in range(250):
            lams2, gams, infos, st = batch.gn_batch_graph_step(lams, gams)
        for f in range(len(fits)):
            r, _ = batch.gn_signed_max_residual(f, thetas[f], lams[f], 0.1)
            hist_r[f].append(r)
            try:
                lams[f] = gn.gn_funnel_next(hist_l[f], hist_r[f], 0.01)
            except gn.GNError:
                pass
            hist_l[f].append(lams[f])
    batch.close()
    assert abs(statistics.median(lams) - 0.5) < 2e-3, hist_l
    assert all(abs(l - 0.5) < 1e-2 for l in lams), hist_l
