"""Pipelined graph step: the Gram in column-major chunks beside the factorisation.

Under GN_PREC_SPLIT_ALL, gn_step_graph computes G's lower tiles column by column in
launches of at most `tiles` tiles, copies each finished 256-column strip into
A = G + gamma I and lets the factorisation start that strip at once.  Only the
schedule changes: every tile, copy and factor kernel computes what it computed
before, so the step must equal the eager gn_step (and the unpipelined graph) bit
for bit, for chunk sizes from one tile (every strip gated separately, many
launches) to the whole triangle in one launch.
"""
import numpy as np
import pytest

from tests.gpu_cases import dev, gpu_problem, host, small

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

SPLIT_ALL = 2


def steps(prob, theta, lam, gam, n, graph):
    out = []
    for _ in range(n):
        f = prob.gn_step_graph if graph else prob.gn_step
        rc, lam, gam, info = f(theta, lam, gam)
        out.append((rc, lam, gam, info))
    return out


def same(a, b):
    for (rc_a, lam_a, gam_a, ia), (rc_b, lam_b, gam_b, ib) in zip(a, b):
        assert rc_a == rc_b
        assert lam_a == lam_b and gam_a == gam_b
        for k in ("n_trials", "chol_retries", "alpha", "gamma_used", "loss_before", "loss_after"):
            assert ia[k] == ib[k], k


@pytest.mark.parametrize("tiles", [1, 5, 7, -1])
@pytest.mark.parametrize("name", ["burgers", "ccf", "ipm"])
def test_pipelined_step_equals_eager(name, tiles):
    w = small(name)
    pe = gpu_problem(w, precision=SPLIT_ALL, n_slices=6)
    pp = gpu_problem(w, precision=SPLIT_ALL, n_slices=6)
    pp.gn_set_pipeline(tiles)
    te, tp = dev(w.theta), dev(w.theta)
    eager = steps(pe, te, w.lam, 1e-4, 4, graph=False)
    piped = steps(pp, tp, w.lam, 1e-4, 4, graph=True)
    same(eager, piped)
    np.testing.assert_array_equal(host(tp), host(te))
    # the graph's event marks time the overlapped phases: the Jacobian and the Gram, and
    # on the capture stream the Jacobian, factorisation, model and line search in sequence
    ph = piped[-1][3]["ms_phase"]
    assert ph[1] > 0 and ph[3] > 0
    assert ph[0] + ph[1] <= ph[6] * 1.001
    assert ph[0] + ph[3] + ph[4] + ph[5] <= ph[6] * 1.001
    pe.close()
    pp.close()


def test_pipeline_off_and_on_agree_and_recapture():
    """Switching the pipeline on a live handle recaptures; all settings give the same steps."""
    w = small("ccf", seed=5)
    runs = []
    prob = gpu_problem(w, precision=SPLIT_ALL, n_slices=6)
    for tiles in (0, 3, -1, 0):
        prob.gn_set_pipeline(tiles)
        theta = dev(w.theta)
        runs.append((steps(prob, theta, w.lam, 1e-4, 3, graph=True), host(theta)))
    for r, th in runs[1:]:
        same(runs[0][0], r)
        np.testing.assert_array_equal(th, runs[0][1])
    prob.close()


def test_pipelined_not_spd_retries():
    """Every factorisation fails with a negative damping: the pipelined step graph fails and
    the solve graph is replayed with damping x10, five times, as gn_step does."""
    w = small("burgers")
    pe = gpu_problem(w, precision=SPLIT_ALL, n_slices=6)
    pp = gpu_problem(w, precision=SPLIT_ALL, n_slices=6)
    pp.gn_set_pipeline(2)
    te, tp = dev(w.theta), dev(w.theta)
    rc_e, lam_e, gam_e, ie = pe.gn_step(te, w.lam, -1e3)
    rc_p, lam_p, gam_p, ip = pp.gn_step_graph(tp, w.lam, -1e3)
    assert rc_e == rc_p == -5
    assert ip["chol_retries"] == ie["chol_retries"] == 5
    assert lam_p == w.lam and gam_p == gam_e
    np.testing.assert_array_equal(host(tp), w.theta)
    # then a normal pipelined step on the same graphs
    a = steps(pe, te, w.lam, 1e-4, 2, graph=False)
    b = steps(pp, tp, w.lam, 1e-4, 2, graph=True)
    same(a, b)
    np.testing.assert_array_equal(host(tp), host(te))
    pe.close()
    pp.close()


def test_set_pipeline_rejects_bad_values():
    from paper_2509_14185_gb300 import gn
    w = small("burgers")
    prob = gpu_problem(w, precision=SPLIT_ALL, n_slices=6)
    with pytest.raises(gn.GNError):
        prob.gn_set_pipeline(-2)
    prob.close()
