"""Lambda strategies on the GPU (Methods, "Identifying Admissible lambda Values") against the
oracle: training at a fixed lambda, the lambda-inference rule at the origin and the funnel
signal r_hat (signed residual of largest magnitude near the origin)."""
import numpy as np
import pytest

from oracle import lam as olam
from tests.gpu_cases import CASES, TOL, dev, gpu_problem, host, oracle_problem, rel, small

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.mark.parametrize("name", list(CASES))
def test_frozen_lambda_step_matches_oracle(name):
    w = small(name)
    p = oracle_problem(w)
    th_o, lam_o, gam_o, info_o = olam.frozen_gn_step(p, w.theta, w.lam, w.gamma)
    prob = gpu_problem(w)
    prob.gn_set_lambda_trainable(False)
    J = host(prob.jacobian(dev(w.theta), w.lam))
    assert np.all(J[:, -1] == 0.0)
    theta = dev(w.theta)
    rc, lam, gam, info = prob.gn_step(theta, w.lam, w.gamma)
    assert rc == info_o["status"]
    assert lam == w.lam
    assert abs(info["loss_before"] - info_o["loss_before"]) <= TOL * info_o["loss_before"]
    if rc == 0:
        assert info["alpha"] == info_o["alpha"]
        assert gam == pytest.approx(gam_o, rel=1e-15)
        cond = np.linalg.cond(info_o["G"] + info_o["gamma_used"] * np.eye(p.P))
        assert rel(w.theta - host(theta), w.theta - th_o) <= max(TOL, 1e-15 * cond)
    prob.close()


@pytest.mark.parametrize("name", ["ccf", "ipm"])
def test_frozen_lambda_graph_equals_eager(name):
    w = small(name)
    pe, pg = gpu_problem(w, precision=2, n_slices=6), gpu_problem(w, precision=2, n_slices=6)
    for pr in (pe, pg):
        pr.gn_set_lambda_trainable(False)
    te, tg = dev(w.theta), dev(w.theta)
    le = lg = w.lam
    ge = gg = 1e-4
    for _ in range(3):
        rc_e, le, ge, _ = pe.gn_step(te, le, ge)
        rc_g, lg, gg, _ = pg.gn_step_graph(tg, lg, gg)
        assert rc_e == rc_g
    assert le == lg == w.lam and ge == gg
    np.testing.assert_array_equal(host(tg), host(te))
    # making lambda trainable again recaptures: both paths move lambda identically
    pe.gn_set_lambda_trainable(True)
    pg.gn_set_lambda_trainable(True)
    rc_e, le2, ge, _ = pe.gn_step(te, le, ge)
    rc_g, lg2, gg, _ = pg.gn_step_graph(tg, lg, gg)
    assert rc_e == rc_g and le2 == lg2 and le2 != w.lam
    pe.close()
    pg.close()


@pytest.mark.parametrize("name", ["ccf", "ipm", "boussinesq"])
def test_lambda_inference_matches_oracle(name):
    w = small(name)
    p = oracle_problem(w)
    th = w.theta + 0.3 * np.sin(np.arange(p.P))
    lam_o = olam.lambda_inference(p, th, w.lam)
    prob = gpu_problem(w)
    lam_g = prob.gn_lambda_inference(dev(th), w.lam)
    base = 3.0 if name == "boussinesq" else 2.0
    assert abs(lam_g - lam_o) <= 1e-12 * max(abs(lam_o), abs(lam_o + base))
    prob.close()


def test_lambda_inference_burgers_is_refused():
    from paper_2509_14185_gb300 import gn
    w = small("burgers")
    prob = gpu_problem(w)
    with pytest.raises(gn.GNError) as e:
        prob.gn_lambda_inference(dev(w.theta), w.lam)
    assert e.value.code == gn.GN_ERR_UNSUPPORTED
    prob.close()


@pytest.mark.parametrize("name", list(CASES))
def test_signed_max_residual_matches_oracle(name):
    w = small(name)
    p = oracle_problem(w)
    r = np.sqrt(np.sum(p.y ** 2, axis=0))
    prob = gpu_problem(w)
    th = dev(w.theta)
    for radius in (np.median(r), 0.3 * np.median(r), np.inf):
        val_o, i_o = olam.signed_max_residual(p, w.theta, w.lam, radius)
        val_g, i_g = prob.gn_signed_max_residual(th, w.lam, radius)
        assert i_g == i_o
        assert abs(val_g - val_o) <= TOL * abs(val_o)
    assert prob.gn_signed_max_residual(th, w.lam, 0.5 * r.min()) == (0.0, -1)
    prob.close()


@pytest.mark.parametrize("name", list(CASES))
def test_field_jets_match_oracle(name):
    """gn_field_jets (the profile and its derivatives at caller points) vs the oracle's fields."""
    w = small(name)
    p = oracle_problem(w)
    prob = gpu_problem(w)
    pts = p.y[:, ::7]
    out = host(prob.gn_field_jets(dev(w.theta), w.lam, pts))
    F = p.fields(w.theta, w.lam, pts, extra_g=(name == "ccf"))
    d, nf = p.d, len(F) - (1 if name == "ccf" else 0)
    nj = 1 + d + (1 if d == 1 else 3)
    for f in range(nf):
        assert rel(out[:, f * nj], F[f].v) <= TOL
        for i in range(d):
            assert rel(out[:, f * nj + 1 + i], F[f].g[i]) <= TOL
        if d == 2:
            for k, (i, j) in enumerate([(0, 0), (0, 1), (1, 1)]):
                assert rel(out[:, f * nj + 3 + k], F[f].h[i][j]) <= TOL
    if name == "ccf":
        assert rel(out[:, nf * nj], F[-1].v) <= TOL
    prob.close()
