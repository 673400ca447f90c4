"""Parity at the benchmark's full size, in the benchmark's launch configuration.

The CCF 1st-unstable workload (16384 points, MLP 1-64-64-64-1, M = 1024
Hilbert nodes, 16385 x 8514 Jacobian) is too large for the oracle's full
complex-step Jacobian, so whole columns are sampled: the oracle computes each
sampled column over all 16385 rows (one complex-step residual pass each) and
the GPU's Jacobian must match them, and the Gram entries between sampled
columns (full-length dot products) must match G from both Gram paths.
"""
import numpy as np
import pytest
import torch

from oracle import gn as ogn
from tests.gpu_cases import TOL, dev, gpu_problem, host, oracle_problem, rel

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def test_ccf_unstable_full_size_sampled_columns_and_gram():
    from paper_2509_14185_gb300 import inputs as I
    w = I.ccf_unstable_1d()
    p = oracle_problem(w)
    cols = [0, 63, 64 + 4096, 4160 + 2000, 8513, p.P]       # first/hidden/output layers and lambda
    Jc = ogn.jacobian(p, w.theta, w.lam, cols)
    r_o = p.rows(w.theta, w.lam)
    from tests.test_gpu_split import split_bound
    Gbound = {0: None, 2: 2.0 * split_bound(Jc, 6)}
    for prec, bound in [(0, TOL), (2, 1e-11)]:
        prob = gpu_problem(w, precision=prec, n_slices=6)
        theta = dev(w.theta)
        r, loss = prob.residual(theta, w.lam)
        assert rel(host(r), r_o) <= TOL
        J = prob.jacobian(theta, w.lam)
        Jh = host(J[:, cols])
        for k in range(len(cols)):
            assert rel(Jh[:, k], Jc[:, k]) <= bound, (prec, cols[k])
        # Gram entries between the sampled columns, from the full Gram of each path
        Pp = prob.P + 1
        G = torch.zeros((Pp, Pp), dtype=torch.float64, device="cuda")
        g = prob.new_vec(Pp)
        prob.gn_gram(J.contiguous(), J.shape[0], r, G, g, precision=max(prec, 0))
        Gh = host(G)
        Gs = Jc.T @ Jc
        for a in range(len(cols)):
            for b in range(a + 1):
                i, j = max(cols[a], cols[b]), min(cols[a], cols[b])
                ref = Gs[a, b]
                scale = np.linalg.norm(Jc[:, a]) * np.linalg.norm(Jc[:, b])
                tol = 1e-12 * scale if prec == 0 else Gbound[prec][a, b] + 1e-12 * scale
                assert abs(Gh[i, j] - ref) <= tol, (prec, cols[a], cols[b])
        assert rel(host(g)[cols], (Jc.T @ r_o)) <= bound
        prob.close()
