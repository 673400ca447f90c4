"""Thin Python binding of libgn (include/gn.h): argument marshalling only.

Every step of the Gauss-Newton path runs in the library's CUDA kernels; this
module converts torch tensors to device pointers and calls the C ABI by the
same names.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the shared library is missing, `lib()` raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

from . import inputs as _inputs

GN_OK = 0
GN_WARN_NO_DECREASE = 1
GN_ERR_INVALID = -1
GN_ERR_CUDA = -2
GN_ERR_OOM = -3
GN_ERR_NONFINITE = -4
GN_ERR_NOT_SPD = -5
GN_ERR_TIMEOUT = -6
GN_ERR_UNSUPPORTED = -7
GN_ERR_TOO_LARGE = -8
GN_ERR_IO = -9
GN_ERR_MISMATCH = -10

GN_PREC_FP64 = 0
GN_PREC_SPLIT_BF16 = 1
GN_PREC_SPLIT_ALL = 2
GN_MAX_LAYERS = 8

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libgn.so")


class gn_problem(ctypes.Structure):
    _fields_ = [
        ("equation", ctypes.c_int),
        ("n_layers", ctypes.c_int),
        ("widths", ctypes.c_int * (GN_MAX_LAYERS + 1)),
        ("n_pts", ctypes.c_int64),
        ("y", ctypes.c_void_p),
        ("rho", ctypes.c_void_p),
        ("n_bnd", ctypes.c_int64),
        ("y_bnd", ctypes.c_void_p),
        ("c_bnd", ctypes.c_double),
        ("y_norm", ctypes.c_double * 2),
        ("c_norm", ctypes.c_double),
        ("c_norm_w", ctypes.c_double),
        ("hilbert_m", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("n_slices", ctypes.c_int),
        ("fourier_m", ctypes.c_int),
        ("fourier_B", ctypes.c_void_p),
        ("n_inf", ctypes.c_int64),
        ("y_inf", ctypes.c_void_p),
        ("c_inf", ctypes.c_double),
        ("norm_kind", ctypes.c_int),
        ("norm_field", ctypes.c_int),
        ("output_map", ctypes.c_int),
        ("row_block", ctypes.c_int64),
        ("n_relu", ctypes.c_int64),
        ("y_relu", ctypes.c_void_p),
        ("c_relu", ctypes.c_double),
        ("relu_bound", ctypes.c_double),
        ("relu_sign", ctypes.c_int),
        ("n_d1", ctypes.c_int64),
        ("y_d1", ctypes.c_void_p),
        ("rho_d1", ctypes.c_void_p),
        ("c_d1", ctypes.c_double),
        ("n_d2", ctypes.c_int64),
        ("y_d2", ctypes.c_void_p),
        ("rho_d2", ctypes.c_void_p),
        ("c_d2", ctypes.c_double),
    ]


class gn_step_info(ctypes.Structure):
    _fields_ = [
        ("loss_before", ctypes.c_double),
        ("loss_after", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("gamma_used", ctypes.c_double),
        ("chol_retries", ctypes.c_int),
        ("n_trials", ctypes.c_int),
        ("status", ctypes.c_int),
        ("ms_phase", ctypes.c_double * 8),
        ("momentum", ctypes.c_double),
        ("max_abs_res", ctypes.c_double),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "ms_phase"}
        d["ms_phase"] = list(self.ms_phase)
        return d


_LIB = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double

EXPORTS = {
    "gn_init": (ctypes.c_int, [ctypes.POINTER(gn_problem), _P, ctypes.POINTER(_P)]),
    "gn_destroy": (ctypes.c_int, [_P]),
    "gn_param_count": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "gn_row_count": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "gn_set_precision": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "gn_residual": (ctypes.c_int, [_P, _P, _D, _P, ctypes.POINTER(_D)]),
    "gn_jacobian": (ctypes.c_int, [_P, _P, _D, _P, _I64, _I64, _I64]),
    "gn_gradient": (ctypes.c_int, [_P, _P, _D, _P, _P]),
    "gn_gram": (ctypes.c_int, [_P, _P, _I64, _I64, _P, _P, _P, ctypes.c_int, ctypes.c_int]),
    "gn_damped_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(_D), _P, ctypes.POINTER(ctypes.c_int)]),
    "gn_step": (ctypes.c_int, [_P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(gn_step_info)]),
    "gn_max_residual": (ctypes.c_int, [_P, _P, _D, ctypes.POINTER(_D)]),
    "gn_step_ema": (ctypes.c_int, [_P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D), _P, _P, _P, _D, ctypes.c_int,
                                   ctypes.POINTER(gn_step_info)]),
    "gn_save": (ctypes.c_int, [_P, ctypes.c_char_p, _P, _D, _D]),
    "gn_load": (ctypes.c_int, [_P, ctypes.c_char_p, _P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "gn_jtr_noalloc": (ctypes.c_int, [_P, _I64, _I64, _I64, _P, _P, _P]),
    "gn_batch_init": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_P)]),
    "gn_batch_handle": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "gn_batch_step": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "gn_batch_destroy": (ctypes.c_int, [_P]),
    "gn_set_gram_split": (ctypes.c_int, [_P, ctypes.c_int]),
    "gn_set_pipeline": (ctypes.c_int, [_P, ctypes.c_int]),
    "gn_pipeline_tiles": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "gn_set_lambda_trainable": (ctypes.c_int, [_P, ctypes.c_int]),
    "gn_set_stage1": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _D, _D]),
    "gn_field_jets": (ctypes.c_int, [_P, _P, _D, _P, _I64, _P]),
    "gn_field_jets_ld": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "gn_lambda_inference": (ctypes.c_int, [_P, _P, _D, ctypes.POINTER(_D)]),
    "gn_signed_max_residual": (ctypes.c_int, [_P, _P, _D, _D, ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    "gn_funnel_next": (ctypes.c_int, [_P, _P, ctypes.c_int, _D, ctypes.POINTER(_D)]),
    "gn_gram_split_choice": (ctypes.c_int, [_P, _I64, ctypes.POINTER(ctypes.c_int)]),
    "gn_set_gram_tile": (ctypes.c_int, [_P, ctypes.c_int]),
    "gn_gram_tile_choice": (ctypes.c_int, [_P, _I64, ctypes.POINTER(ctypes.c_int)]),
    "gn_step_graph": (ctypes.c_int, [_P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(gn_step_info)]),
    "gn_batch_capture_graph": (ctypes.c_int, [_P, _P]),
    "gn_batch_graph_step": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "gn_test_bounded_waits": (ctypes.c_int, [ctypes.c_ulonglong, ctypes.c_int]),
    "gn_kernel_launches": (ctypes.c_int64, []),
    "gn_last_error_detail": (ctypes.c_char_p, []),
    "gn_error_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def lib():
    """Load libgn.so (built in-tree by paper_2509_14185_gb300.build)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgn.so is not built ({LIB_PATH}); run paper_2509_14185_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class GNError(RuntimeError):
    def __init__(self, code, where):
        msg = lib().gn_error_string(code).decode()
        detail = lib().gn_last_error_detail().decode()
        super().__init__(f"{where}: {msg} ({code})" + (f" [{detail}]" if detail else ""))
        self.code = code


def _check(code, where):
    if code < 0:
        raise GNError(code, where)
    return code


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), "expected a contiguous cuda float64 tensor"
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class GNProblem:
    """One profile fit bound to a libgn handle (device memory owned by torch and libgn)."""

    def __init__(self, equation, widths, y, y_bnd=None, rho=None, c_bnd=1.0, y_norm=(1.0, 0.0), c_norm=1.0,
                 c_norm_w=1.0, hilbert_m=1024, precision=GN_PREC_FP64, n_slices=4, device="cuda", stream=None,
                 fourier_B=None, y_inf=None, c_inf=1.0, norm_field=None, norm_deriv=None, output_map=0,
                 row_block=0, y_relu=None, c_relu=1.0, relu_bound=0.0, relu_sign=1,
                 y_d1=None, rho_d1=None, c_d1=1.0, y_d2=None, rho_d2=None, c_d2=1.0):
        lib()
        self.device = torch.device(device)
        self.equation = int(equation)
        self.widths = list(widths)
        self.d = _inputs.EQUATION_DIM[self.equation]
        y = np.asarray(y, dtype=np.float64).reshape(self.d, -1)
        self.y = torch.from_numpy(np.ascontiguousarray(y)).to(self.device)
        self.n_pts = y.shape[1]
        yb = np.zeros((self.d, 0)) if y_bnd is None else np.asarray(y_bnd, dtype=np.float64).reshape(self.d, -1)
        self.y_bnd = torch.from_numpy(np.ascontiguousarray(yb)).to(self.device) if yb.size else None
        self.n_bnd = yb.shape[1] if yb.size else 0
        self.rho = None if rho is None else torch.as_tensor(rho, dtype=torch.float64, device=self.device).contiguous()
        # decay points of the data loss (SoA [d][n_inf]); rows after the wall rows
        yi = np.zeros((self.d, 0)) if y_inf is None else np.asarray(y_inf, dtype=np.float64).reshape(self.d, -1)
        self.y_inf = torch.from_numpy(np.ascontiguousarray(yi)).to(self.device) if yi.size else None
        self.n_inf = yi.shape[1] if yi.size else 0
        p = gn_problem()
        p.equation = self.equation
        p.n_layers = len(self.widths) - 1
        for i, w in enumerate(self.widths):
            p.widths[i] = int(w)
        p.n_pts = self.n_pts
        p.y = self.y.data_ptr() if self.n_pts else None
        p.rho = self.rho.data_ptr() if self.rho is not None else None
        p.n_bnd = self.n_bnd
        p.y_bnd = self.y_bnd.data_ptr() if self.y_bnd is not None else None
        p.c_bnd = float(c_bnd)
        p.y_norm[0], p.y_norm[1] = float(y_norm[0]), float(y_norm[1])
        p.c_norm = float(c_norm)
        p.c_norm_w = float(c_norm_w)
        p.hilbert_m = int(hilbert_m)
        p.precision = int(precision)
        p.n_slices = int(n_slices)
        p.n_inf = self.n_inf
        p.y_inf = self.y_inf.data_ptr() if self.y_inf is not None else None
        p.c_inf = float(c_inf)
        p.output_map = int(output_map)   # 0 linear, 1 exp
        p.row_block = int(row_block)     # 0: automatic
        # bound points of the data loss (SoA [d][n_relu]); rows after the decay rows
        yr = np.zeros((self.d, 0)) if y_relu is None else np.asarray(y_relu, dtype=np.float64).reshape(self.d, -1)
        self.y_relu = torch.from_numpy(np.ascontiguousarray(yr)).to(self.device) if yr.size else None
        p.n_relu = yr.shape[1] if yr.size else 0
        p.y_relu = self.y_relu.data_ptr() if self.y_relu is not None else None
        p.c_relu, p.relu_bound, p.relu_sign = float(c_relu), float(relu_bound), int(relu_sign)
        # derivative-loss batches (SoA [d][n]); their rows follow the interior rows
        self._dkeep = []
        for k, (yd, rd, cd) in enumerate(((y_d1, rho_d1, c_d1), (y_d2, rho_d2, c_d2))):
            ya = np.zeros((self.d, 0)) if yd is None else np.asarray(yd, dtype=np.float64).reshape(self.d, -1)
            nd = ya.shape[1] if ya.size else 0
            yt = torch.from_numpy(np.ascontiguousarray(ya)).to(self.device) if nd else None
            rt = (None if rd is None or not nd
                  else torch.as_tensor(rd, dtype=torch.float64, device=self.device).contiguous())
            self._dkeep += [yt, rt]
            setattr(p, f"n_d{k + 1}", nd)
            setattr(p, f"y_d{k + 1}", yt.data_ptr() if yt is not None else None)
            setattr(p, f"rho_d{k + 1}", rt.data_ptr() if rt is not None else None)
            setattr(p, f"c_d{k + 1}", float(cd))
        # normalisation constraint: the equation's own unless a field or derivative is given
        if norm_field is not None or norm_deriv is not None:
            deriv = (self.equation == _inputs.BOUSSINESQ) if norm_deriv is None else bool(norm_deriv)
            p.norm_kind = 2 if deriv else 1
            p.norm_field = 0 if norm_field is None else int(norm_field)
        if fourier_B is not None:
            # host copy kept alive for gn_init (which copies it)
            self._fourier_B = np.ascontiguousarray(np.asarray(fourier_B, dtype=np.float64))
            p.fourier_m = int(self._fourier_B.shape[0])
            p.fourier_B = self._fourier_B.ctypes.data
        self._prob = p
        self.stream = stream
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().gn_init(ctypes.byref(p), _stream_ptr(stream), ctypes.byref(h)), "gn_init")
        self.h = h
        P = _I64()
        _check(lib().gn_param_count(h, ctypes.byref(P)), "gn_param_count")
        R = _I64()
        _check(lib().gn_row_count(h, ctypes.byref(R)), "gn_row_count")
        self.P, self.n_rows = P.value, R.value

    @classmethod
    def from_workload(cls, w, **kw):
        kw.setdefault("y_inf", getattr(w, "y_inf", None))
        kw.setdefault("c_inf", getattr(w, "c_inf", 1.0))
        kw.setdefault("norm_field", getattr(w, "norm_field", None))
        kw.setdefault("norm_deriv", getattr(w, "norm_deriv", None))
        kw.setdefault("output_map", getattr(w, "output_map", 0))
        kw.setdefault("c_bnd", getattr(w, "c_bnd", 1.0))
        for k, dflt in (("y_d1", None), ("rho_d1", None), ("c_d1", 1.0), ("y_d2", None), ("rho_d2", None),
                        ("c_d2", 1.0)):
            kw.setdefault(k, getattr(w, k, dflt))
        kw.setdefault("c_norm_w", getattr(w, "c_norm_w", 1.0))
        for k, dflt in (("y_relu", None), ("c_relu", 1.0), ("relu_bound", 0.0), ("relu_sign", 1)):
            kw.setdefault(k, getattr(w, k, dflt))
        return cls(w.equation, w.widths, w.y, w.y_bnd if w.y_bnd.size else None, w.rho, y_norm=w.y_norm,
                   c_norm=w.c_norm, hilbert_m=w.hilbert_m, **kw)

    def close(self):
        if getattr(self, "h", None):
            lib().gn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls with the C names ------------------------------------------------
    def gn_set_precision(self, precision, n_slices=0):
        _check(lib().gn_set_precision(self.h, int(precision), int(n_slices)), "gn_set_precision")

    def gn_set_gram_split(self, ksplit):
        _check(lib().gn_set_gram_split(self.h, int(ksplit)), "gn_set_gram_split")

    def gn_set_gram_tile(self, tile_n):
        """Split Gram output tiles 128 x tile_n (128 or 64; 0: autotuned)."""
        _check(lib().gn_set_gram_tile(self.h, int(tile_n)), "gn_set_gram_tile")

    def gn_gram_tile_choice(self, nrows=None):
        k = ctypes.c_int(0)
        _check(lib().gn_gram_tile_choice(self.h, self.n_rows if nrows is None else int(nrows), ctypes.byref(k)),
               "gn_gram_tile_choice")
        return k.value

    def gn_set_pipeline(self, tiles):
        """Tiles per Gram chunk of the pipelined graph step (0, the default: off; -1: from the SM count)."""
        _check(lib().gn_set_pipeline(self.h, int(tiles)), "gn_set_pipeline")

    def gn_pipeline_tiles(self):
        """Tiles per Gram chunk of the next captured step (0: that step is not pipelined)."""
        t = _I64(0)
        _check(lib().gn_pipeline_tiles(self.h, ctypes.byref(t)), "gn_pipeline_tiles")
        return int(t.value)

    def gn_gram_split_choice(self, nrows=None):
        k = ctypes.c_int(0)
        _check(lib().gn_gram_split_choice(self.h, self.n_rows if nrows is None else int(nrows), ctypes.byref(k)),
               "gn_gram_split_choice")
        return k.value

    def gn_set_lambda_trainable(self, trainable):
        _check(lib().gn_set_lambda_trainable(self.h, int(bool(trainable))), "gn_set_lambda_trainable")

    def gn_set_stage1(self, widths1, theta1, lam, eps):
        """Make this problem the second stage of a fit whose first stage is (widths1, theta1)."""
        w = (ctypes.c_int * len(widths1))(*[int(v) for v in widths1])
        _check(lib().gn_set_stage1(self.h, len(widths1) - 1, w, _ptr(theta1), float(lam), float(eps)),
               "gn_set_stage1")

    def gn_field_jets(self, theta, lam, y):
        """Field jets of the handle's network at points y (d, n): a device tensor (n, ld)."""
        y = torch.as_tensor(np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(self.d, -1)),
                            device=self.device)
        ld = _I64()
        _check(lib().gn_field_jets_ld(self.h, ctypes.byref(ld)), "gn_field_jets_ld")
        out = torch.empty((y.shape[1], ld.value), dtype=torch.float64, device=self.device)
        _check(lib().gn_field_jets(self.h, _ptr(theta), float(lam), _ptr(y), y.shape[1], _ptr(out)),
               "gn_field_jets")
        torch.cuda.synchronize(self.device)
        return out

    def gn_lambda_inference(self, theta, lam):
        out = _D()
        _check(lib().gn_lambda_inference(self.h, _ptr(theta), float(lam), ctypes.byref(out)), "gn_lambda_inference")
        return out.value

    def gn_signed_max_residual(self, theta, lam, radius):
        out = _D()
        idx = _I64()
        _check(lib().gn_signed_max_residual(self.h, _ptr(theta), float(lam), float(radius), ctypes.byref(out),
                                            ctypes.byref(idx)), "gn_signed_max_residual")
        return out.value, idx.value

    def gn_residual(self, theta, lam, r_out=None, want_loss=True):
        loss = _D()
        rc = lib().gn_residual(self.h, _ptr(theta), float(lam), _ptr(r_out),
                               ctypes.byref(loss) if want_loss else None)
        if rc == GN_ERR_NONFINITE:
            return rc, loss.value
        _check(rc, "gn_residual")
        return rc, loss.value

    def gn_jacobian(self, theta, lam, J_out, row0=0, nrows=None):
        nrows = self.n_rows - row0 if nrows is None else nrows
        _check(lib().gn_jacobian(self.h, _ptr(theta), float(lam), _ptr(J_out), J_out.stride(0), row0, nrows),
               "gn_jacobian")

    def gn_gradient(self, theta, lam, seed, grad_out):
        _check(lib().gn_gradient(self.h, _ptr(theta), float(lam), _ptr(seed), _ptr(grad_out)), "gn_gradient")

    def gn_gram(self, J, nrows, r, G_out, g_out, precision=GN_PREC_FP64, accumulate=False):
        _check(lib().gn_gram(self.h, _ptr(J), J.stride(0), int(nrows), _ptr(r), _ptr(G_out), _ptr(g_out),
                             int(precision), int(bool(accumulate))), "gn_gram")

    def gn_damped_solve(self, G, g, gamma, delta_out):
        gam = _D(gamma)
        ret = ctypes.c_int(0)
        rc = lib().gn_damped_solve(self.h, _ptr(G), _ptr(g), ctypes.byref(gam), _ptr(delta_out), ctypes.byref(ret))
        return rc, gam.value, ret.value

    def gn_step(self, theta, lam, gamma):
        lam_ = _D(lam)
        gam_ = _D(gamma)
        info = gn_step_info()
        rc = lib().gn_step(self.h, _ptr(theta), ctypes.byref(lam_), ctypes.byref(gam_), ctypes.byref(info))
        if rc < 0 and rc not in (GN_ERR_NOT_SPD, GN_ERR_NONFINITE):
            _check(rc, "gn_step")
        return rc, lam_.value, gam_.value, info.as_dict()

    def gn_step_graph(self, theta, lam, gamma):
        """gn_step through the handle's captured CUDA graphs (captured on the first call for theta)."""
        lam_ = _D(lam)
        gam_ = _D(gamma)
        info = gn_step_info()
        rc = lib().gn_step_graph(self.h, _ptr(theta), ctypes.byref(lam_), ctypes.byref(gam_), ctypes.byref(info))
        if rc < 0 and rc not in (GN_ERR_NOT_SPD, GN_ERR_NONFINITE):
            _check(rc, "gn_step_graph")
        return rc, lam_.value, gam_.value, info.as_dict()

    def gn_step_ema(self, theta, lam, gamma, G_ema, v_prev, signs, beta, first):
        """The paper's EMA rank-1 optimiser: theta, G_ema, v_prev updated in place."""
        lam_ = _D(lam)
        gam_ = _D(gamma)
        info = gn_step_info()
        rc = lib().gn_step_ema(self.h, _ptr(theta), ctypes.byref(lam_), ctypes.byref(gam_), _ptr(G_ema),
                               _ptr(v_prev), _ptr(signs), float(beta), int(bool(first)), ctypes.byref(info))
        if rc < 0 and rc not in (GN_ERR_NOT_SPD, GN_ERR_NONFINITE):
            _check(rc, "gn_step_ema")
        return rc, lam_.value, gam_.value, info.as_dict()

    def gn_max_residual(self, theta, lam):
        out = _D()
        _check(lib().gn_max_residual(self.h, _ptr(theta), float(lam), ctypes.byref(out)), "gn_max_residual")
        return out.value

    def gn_save(self, path, theta, lam, gamma):
        _check(lib().gn_save(self.h, os.fsencode(path), _ptr(theta), float(lam), float(gamma)), "gn_save")

    def gn_load(self, path, theta_out):
        lam, gam = _D(), _D()
        _check(lib().gn_load(self.h, os.fsencode(path), _ptr(theta_out), ctypes.byref(lam), ctypes.byref(gam)),
               "gn_load")
        return lam.value, gam.value

    # -- conveniences --------------------------------------------------------------
    def new_vec(self, n):
        return torch.zeros(n, dtype=torch.float64, device=self.device)

    def residual(self, theta, lam):
        r = self.new_vec(self.n_rows)
        rc, loss = self.gn_residual(theta, lam, r)
        return r, loss

    def jacobian(self, theta, lam, row0=0, nrows=None, ld=None):
        nrows = self.n_rows - row0 if nrows is None else nrows
        ld = self.P + 1 if ld is None else ld
        J = torch.zeros((nrows, ld), dtype=torch.float64, device=self.device)
        self.gn_jacobian(theta, lam, J, row0, nrows)
        return J[:, : self.P + 1]

    def gradient(self, theta, lam, seed=None):
        g = self.new_vec(self.P + 1)
        self.gn_gradient(theta, lam, seed, g)
        return g


def gn_funnel_next(lambdas, r_hats, dlambda):
    """Next lambda of funnel inference (secant on the last two (lambda, r_hat) pairs)."""
    n = len(lambdas)
    la = (ctypes.c_double * max(1, n))(*lambdas)
    ra = (ctypes.c_double * max(1, n))(*r_hats)
    out = _D()
    _check(lib().gn_funnel_next(la, ra, int(n), float(dlambda), ctypes.byref(out)), "gn_funnel_next")
    return out.value


class ResidualFn(torch.autograd.Function):
    """r~(theta, lambda) as a differentiable torch op: forward calls gn_residual, backward
    calls the adjoint kernel gn_gradient seeded by the incoming gradient (the same
    reverse pass that produces the Gauss-Newton Jacobian rows)."""

    @staticmethod
    def forward(ctx, theta, lam, prob: GNProblem):
        r = prob.new_vec(prob.n_rows)
        prob.gn_residual(theta.detach().contiguous(), float(lam), r, want_loss=False)
        ctx.prob = prob
        ctx.save_for_backward(theta.detach(), lam.detach())
        return r

    @staticmethod
    def backward(ctx, grad_r):
        theta, lam = ctx.saved_tensors
        prob = ctx.prob
        g = prob.gradient(theta.contiguous(), float(lam), grad_r.contiguous())
        return g[: prob.P], g[prob.P].reshape(lam.shape), None


def residual_fn(theta, lam, prob):
    return ResidualFn.apply(theta, lam, prob)


class GNBatch:
    """Many independent profile fits stepped together (gn_batch_*): each fit keeps its
    own libgn handle; fits are spread over `n_streams` CUDA streams."""

    def __init__(self, workloads, n_streams=8, precision=GN_PREC_FP64, n_slices=6, device="cuda"):
        lib()
        self.device = torch.device(device)
        self.keep = []
        probs = (gn_problem * len(workloads))()
        for k, w in enumerate(workloads):
            d = _inputs.EQUATION_DIM[w.equation]
            y = torch.from_numpy(np.ascontiguousarray(np.asarray(w.y, dtype=np.float64).reshape(d, -1))).to(self.device)
            yb = None
            if w.y_bnd.size:
                yb = torch.from_numpy(np.ascontiguousarray(w.y_bnd)).to(self.device)
            rho = None if w.rho is None else torch.as_tensor(w.rho, dtype=torch.float64,
                                                             device=self.device).contiguous()
            self.keep += [y, yb, rho]
            p = probs[k]
            p.equation = w.equation
            p.n_layers = len(w.widths) - 1
            for i, wd in enumerate(w.widths):
                p.widths[i] = int(wd)
            p.n_pts = y.shape[1]
            p.y = y.data_ptr()
            p.rho = None if rho is None else rho.data_ptr()
            p.n_bnd = 0 if yb is None else yb.shape[1]
            p.y_bnd = None if yb is None else yb.data_ptr()
            p.c_bnd = 1.0
            p.y_norm[0], p.y_norm[1] = float(w.y_norm[0]), float(w.y_norm[1])
            p.c_norm = float(w.c_norm)
            p.c_norm_w = 1.0
            p.hilbert_m = int(w.hilbert_m)
            p.precision = int(precision)
            p.n_slices = int(n_slices)
        self._probs = probs
        b = ctypes.c_void_p()
        _check(lib().gn_batch_init(probs, len(workloads), int(n_streams), ctypes.byref(b)), "gn_batch_init")
        self.b = b
        self.n = len(workloads)
        self.P = []
        for f in range(self.n):
            h = ctypes.c_void_p()
            _check(lib().gn_batch_handle(b, f, ctypes.byref(h)), "gn_batch_handle")
            P = _I64()
            lib().gn_param_count(h, ctypes.byref(P))
            self.P.append(P.value)

    def gn_batch_step(self, thetas, lambdas, dampings):
        """thetas: list of device tensors (updated in place); lambdas, dampings: lists (returned updated)."""
        ptrs = (ctypes.c_void_p * self.n)(*[t.data_ptr() for t in thetas])
        lam = (ctypes.c_double * self.n)(*lambdas)
        gam = (ctypes.c_double * self.n)(*dampings)
        infos = (gn_step_info * self.n)()
        st = (ctypes.c_int * self.n)()
        torch.cuda.synchronize(self.device)     # the batch's streams do not wait on torch's
        rc = lib().gn_batch_step(self.b, ptrs, lam, gam, infos, st)
        _check(rc if rc < 0 and rc not in (GN_ERR_NOT_SPD, GN_ERR_NONFINITE) else 0, "gn_batch_step")
        return list(lam), list(gam), [infos[i].as_dict() for i in range(self.n)], list(st)

    def handle(self, f):
        h = ctypes.c_void_p()
        _check(lib().gn_batch_handle(self.b, int(f), ctypes.byref(h)), "gn_batch_handle")
        return h

    def gn_set_lambda_trainable(self, trainable):
        """Hold lambda fixed (False) or train it (True) in every fit (capture graphs after this)."""
        for f in range(self.n):
            _check(lib().gn_set_lambda_trainable(self.handle(f), int(bool(trainable))), "gn_set_lambda_trainable")

    def gn_signed_max_residual(self, f, theta, lam, radius):
        out = _D()
        idx = _I64()
        torch.cuda.synchronize(self.device)
        _check(lib().gn_signed_max_residual(self.handle(f), _ptr(theta), float(lam), float(radius),
                                            ctypes.byref(out), ctypes.byref(idx)), "gn_signed_max_residual")
        return out.value, idx.value

    def gn_batch_capture_graph(self, thetas):
        """Capture every fit's step into one CUDA graph for these parameter tensors."""
        self._graph_thetas = list(thetas)
        ptrs = (ctypes.c_void_p * self.n)(*[t.data_ptr() for t in thetas])
        torch.cuda.synchronize(self.device)
        _check(lib().gn_batch_capture_graph(self.b, ptrs), "gn_batch_capture_graph")

    def gn_batch_graph_step(self, lambdas, dampings):
        """One step of every fit as one graph launch (on the tensors given to gn_batch_capture_graph)."""
        lam = (ctypes.c_double * self.n)(*lambdas)
        gam = (ctypes.c_double * self.n)(*dampings)
        infos = (gn_step_info * self.n)()
        st = (ctypes.c_int * self.n)()
        torch.cuda.synchronize(self.device)
        rc = lib().gn_batch_graph_step(self.b, lam, gam, infos, st)
        _check(rc if rc < 0 and rc not in (GN_ERR_NOT_SPD, GN_ERR_NONFINITE) else 0, "gn_batch_graph_step")
        return list(lam), list(gam), [infos[i].as_dict() for i in range(self.n)], list(st)

    def close(self):
        if getattr(self, "b", None):
            lib().gn_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
