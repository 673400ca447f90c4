"""Parity at full size for the 2D configurations: IPM with boundary (65536 points +
4096 wall points, MLP 2-64x4-2, 135169 x 12803 Jacobian) and Boussinesq with
boundary (262144 + 16384 points, MLP 2-128x4-3, 802817 x 50308 Jacobian, 323 GB,
streamed in row blocks).

The oracle cannot evaluate whole columns at these sizes in test time (one
complex-step Boussinesq column is about a minute), but in 2D every row belongs
to one point, so the oracle evaluates a subset of the points, with the loss
weights rescaled (rho and c_bnd by N_sub / N) so that each row carries exactly
the weight it has in the full problem.  The GPU Jacobian is produced at full
size in the library's row blocks; sampled columns are compared on the sampled
rows.  The split Gram entries between the sampled columns are compared with
FP64 dot products of the GPU's full columns (within the split error bound).
"""
import numpy as np
import pytest
import torch

from oracle import gn as ogn
from oracle import problems as Pb
from tests.gpu_cases import TOL, dev, host, rel

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

BLOCK = 16384   # rows per Jacobian block fetched from the library


def subset_oracle(w, pts, walls):
    n, nb = w.y.shape[1], w.y_bnd.shape[1]
    rho = np.full(len(pts), len(pts) / n)
    return Pb.Problem(w.equation, w.widths, w.y[:, pts], w.y_bnd[:, walls], rho, c_bnd=len(walls) / nb,
                      y_norm=w.y_norm, c_norm=w.c_norm, hilbert_m=w.hilbert_m)


def full_rows(w, ne, pts, walls):
    n = w.y.shape[1]
    inner = (np.asarray(pts)[:, None] * ne + np.arange(ne)[None, :]).reshape(-1)
    return np.concatenate([inner, n * ne + np.asarray(walls), [n * ne + w.y_bnd.shape[1]]])


@pytest.mark.parametrize("name", ["ipm", "boussinesq"])
def test_2d_full_size_sampled(name):
    from paper_2509_14185_gb300 import gn
    from paper_2509_14185_gb300 import inputs as I
    from tests.test_gpu_split import split_bound
    w = I.WORKLOADS[name]()
    ne = I.EQUATION_FIELDS[w.equation]
    rng = np.random.default_rng(7)
    pts = np.sort(rng.choice(w.y.shape[1], 384, replace=False))
    walls = np.sort(rng.choice(w.y_bnd.shape[1], 48, replace=False))
    po = subset_oracle(w, pts, walls)
    rows = full_rows(w, ne, pts, walls)
    P = po.P
    cols = [0, 7, P // 3, P // 2, P - 3, P - 1, P]   # first / middle / output layers and lambda
    J_o = ogn.jacobian(po, w.theta, w.lam, cols)
    r_o = po.rows(w.theta, w.lam)

    prob = gn.GNProblem.from_workload(w, precision=gn.GN_PREC_SPLIT_ALL, n_slices=6)
    assert prob.n_rows == rows[-1] + 1 and prob.P == P
    theta = dev(w.theta)
    r, loss = prob.residual(theta, w.lam)
    assert rel(host(r)[rows], r_o) <= TOL
    # Jacobian in row blocks: sampled columns over all rows, and the split Gram accumulated
    Pp = P + 1
    ld = (Pp + 15) // 16 * 16
    Jb = torch.empty((BLOCK, ld), dtype=torch.float64, device="cuda")
    Jc = np.zeros((prob.n_rows, len(cols)))
    G = torch.zeros((Pp, Pp), dtype=torch.float64, device="cuda")
    g = prob.new_vec(Pp)
    ci = torch.tensor(cols, device="cuda")
    for b0 in range(0, prob.n_rows, BLOCK):
        nr = min(BLOCK, prob.n_rows - b0)
        prob.gn_jacobian(theta, w.lam, Jb, row0=b0, nrows=nr)
        Jc[b0:b0 + nr] = host(Jb[:nr].index_select(1, ci))
        prob.gn_gram(Jb, nr, r[b0:b0 + nr], G, g, precision=gn.GN_PREC_SPLIT_BF16, accumulate=b0 > 0)
    for k, c in enumerate(cols):
        assert rel(Jc[rows, k], J_o[:, k]) <= TOL, (name, c)
    # Gram and gradient at full size (the reference is the FP64 product of the GPU's own full columns,
    # whose sampled rows were just checked against the oracle)
    Gh = host(G)
    bound = split_bound(Jc, 6)
    Gs = Jc.T @ Jc
    for a in range(len(cols)):
        for b in range(a + 1):
            i, j = max(cols[a], cols[b]), min(cols[a], cols[b])
            scale = np.linalg.norm(Jc[:, a]) * np.linalg.norm(Jc[:, b])
            assert abs(Gh[i, j] - Gs[a, b]) <= 2.0 * bound[a, b] + 1e-12 * scale, (name, cols[a], cols[b])
    assert rel(host(g)[cols], Jc.T @ host(r)) <= 1e-12
    prob.close()
