"""Checkpoint and resume (gn_save / gn_load): a fit saved after some Gauss-Newton
steps and loaded into a fresh handle continues exactly as the uninterrupted fit
(every reduction in the library has a fixed order); files of another
architecture are refused."""
import numpy as np
import pytest
import torch

from tests.gpu_cases import dev, gpu_problem, host, small

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def test_save_load_resume(tmp_path):
    from paper_2509_14185_gb300 import gn
    w = small("ccf")
    path = tmp_path / "fit.gnck"
    a = gpu_problem(w, precision=gn.GN_PREC_SPLIT_ALL, n_slices=6)
    th = dev(w.theta)
    lam, gam = w.lam, w.gamma
    for _ in range(2):
        _, lam, gam, _ = a.gn_step(th, lam, gam)
    a.gn_save(str(path), th, lam, gam)
    for _ in range(2):
        _, lam, gam, _ = a.gn_step(th, lam, gam)
    b = gpu_problem(w, precision=gn.GN_PREC_SPLIT_ALL, n_slices=6)
    th2 = torch.zeros_like(th)
    lam2, gam2 = b.gn_load(str(path), th2)
    for _ in range(2):
        _, lam2, gam2, _ = b.gn_step(th2, lam2, gam2)
    assert np.array_equal(host(th), host(th2)) and lam == lam2 and gam == gam2
    a.close()
    b.close()


def test_load_refuses_other_architecture(tmp_path):
    from paper_2509_14185_gb300 import gn
    from paper_2509_14185_gb300 import inputs as I
    w = small("ccf")
    path = tmp_path / "fit.gnck"
    a = gpu_problem(w)
    a.gn_save(str(path), dev(w.theta), w.lam, w.gamma)
    other = I.small_case(I.CCF, [1, 12, 12, 1], 40, seed=3, m=32)
    b = gpu_problem(other)
    with pytest.raises(gn.GNError) as e:
        b.gn_load(str(path), torch.zeros(b.P, dtype=torch.float64, device="cuda"))
    assert e.value.code == gn.GN_ERR_MISMATCH
    with pytest.raises(gn.GNError) as e:
        a.gn_load(str(tmp_path / "missing.gnck"), torch.zeros(a.P, dtype=torch.float64, device="cuda"))
    assert e.value.code == gn.GN_ERR_IO
    a.close()
    b.close()
