"""Shared helpers of the GPU parity tests: build the oracle problem and the
libgn problem from the same seeded workload, and the normwise parity metric.

Parity metric (FP64 path): rel(X) = |X_gpu - X_oracle|_inf / |X_oracle|_inf,
and for J also per column.  Bound 1e-12: both sides are FP64 with different
operation orders (reverse-mode jets on the GPU, complex-step forward mode in
the oracle) and different libm implementations of tanh/pow/log.
"""
import numpy as np
import torch

from oracle import gn as ogn
from oracle import problems as Pb
from paper_2509_14185_gb300 import inputs as I

TOL = 1e-12


def oracle_problem(w):
    return Pb.Problem(w.equation, w.widths, w.y, w.y_bnd if w.y_bnd.size else None, w.rho,
                      c_bnd=getattr(w, "c_bnd", 1.0), c_norm_w=getattr(w, "c_norm_w", 1.0),
                      y_norm=w.y_norm, c_norm=w.c_norm, hilbert_m=w.hilbert_m,
                      y_inf=getattr(w, "y_inf", None), c_inf=getattr(w, "c_inf", 1.0),
                      norm_field=getattr(w, "norm_field", None), norm_deriv=getattr(w, "norm_deriv", None),
                      output_map=getattr(w, "output_map", 0), y_relu=getattr(w, "y_relu", None),
                      c_relu=getattr(w, "c_relu", 1.0), relu_bound=getattr(w, "relu_bound", 0.0),
                      relu_sign=getattr(w, "relu_sign", 1),
                      y_d1=getattr(w, "y_d1", None), rho_d1=getattr(w, "rho_d1", None), c_d1=getattr(w, "c_d1", 1.0),
                      y_d2=getattr(w, "y_d2", None), rho_d2=getattr(w, "rho_d2", None), c_d2=getattr(w, "c_d2", 1.0))


def gpu_problem(w, **kw):
    from paper_2509_14185_gb300 import gn
    return gn.GNProblem.from_workload(w, **kw)


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / den) if den > 0 else float(np.max(np.abs(a)))


def col_rel(A, B, floor=0.0):
    """max over columns of |dA_j|_inf / |B_j|_inf (columns whose norm is above floor)."""
    num = np.max(np.abs(A - B), axis=0)
    den = np.max(np.abs(B), axis=0)
    m = den > floor
    return float(np.max(num[m] / den[m])) if np.any(m) else 0.0


CASES = {
    # equation: (widths, n_pts, n_bnd, hilbert M): sizes span several warps / GEMM tiles
    # with ragged tails, small enough for the complex-step oracle to finish in seconds
    "burgers": (I.BURGERS, [1, 24, 24, 1], 203, 0, 64),
    "ccf": (I.CCF, [1, 40, 40, 1], 301, 0, 64),
    "ipm": (I.IPM, [2, 20, 20, 2], 150, 37, 64),
    "boussinesq": (I.BOUSSINESQ, [2, 16, 16, 3], 120, 29, 64),
}


def small(name, seed=11):
    eq, widths, n, nb, m = CASES[name]
    return I.small_case(eq, widths, n, n_bnd=nb, seed=seed, m=m)


def small_weighted(name, seed=11):
    """The same case with non-uniform rho and non-unit wall and normalisation weights."""
    return I.weighted(small(name, seed))
