"""gn_jtr_noalloc: the allocation-free J^T r entry point.

It serves callers that cannot call cudaMalloc (a host application that owns
all device memory through its own allocator, loops that must avoid the
synchronisation an allocation may imply, plug-ins that only receive device
pointers).  Its scratch is a fixed device array in the library image, so the
test checks that two calls in a row (different sizes and data, same shared
scratch) each match the handle-based gn_gram gradient and J^T r formed on the
host in FP64, and that a size beyond the array is rejected.  The file is named
to be collected last; it passes alone in a fresh process and after the other
tests.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _call(L, J, nrows, ncols, r, g):
    return L.gn_jtr_noalloc(ctypes.c_void_p(J.data_ptr()), J.stride(0), nrows, ncols,
                            ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_jtr_matches_gram_gradient_twice():
    from paper_2509_14185_gb300 import build, gn, inputs
    build.build()
    L = gn.lib()
    w = inputs.small_case(inputs.CCF, [1, 24, 24, 1], 180, seed=21, m=32)
    prob = gn.GNProblem.from_workload(w)
    theta = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    J = torch.zeros((prob.n_rows, prob.P + 7), dtype=torch.float64, device="cuda")
    prob.gn_jacobian(theta, w.lam, J)
    Pp = prob.P + 1
    rng = np.random.default_rng(3)
    for nrows in (prob.n_rows, prob.n_rows // 2 + 3):        # two calls in a row, different sizes
        r = torch.tensor(rng.standard_normal(nrows), dtype=torch.float64, device="cuda")
        Jb = J[:nrows]
        G = torch.zeros((Pp, Pp), dtype=torch.float64, device="cuda")
        g_ref = torch.zeros(Pp, dtype=torch.float64, device="cuda")
        prob.gn_gram(Jb, nrows, r, G, g_ref)
        g = torch.full((Pp,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(L, Jb, nrows, Pp, r, g) == gn.GN_OK
        torch.cuda.synchronize()
        ref = g_ref.cpu().numpy()
        got = g.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))
        # and against J^T r formed on the host in FP64 from the same buffers
        host_ref = Jb[:, :Pp].cpu().numpy().T @ r.cpu().numpy()
        assert np.max(np.abs(got - host_ref)) <= TOL * np.max(np.abs(host_ref))
    prob.close()


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    from paper_2509_14185_gb300 import gn
    L = gn.lib()
    J = torch.zeros((2, 16385), dtype=torch.float64, device="cuda")
    r = torch.zeros(2, dtype=torch.float64, device="cuda")
    g = torch.zeros(16385, dtype=torch.float64, device="cuda")
    assert _call(L, J, 2, 16385, r, g) == gn.GN_ERR_TOO_LARGE
    assert L.gn_jtr_noalloc(None, 1, 1, 1, None, None, None) == gn.GN_ERR_INVALID
