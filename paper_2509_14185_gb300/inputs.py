"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module only draws numbers: collocation points, boundary points, initial
network weights and lambda seeds.  It holds none of the method's arithmetic
(no jets, residuals, Gram products or solves), so both the CUDA library and
the CPU oracle can consume its output without sharing any of the computation
that is being checked.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in counter mode: draw i of
stream `seed` is mix(seed + (i+1) * golden_gamma).  Normal deviates use the
Box-Muller transform (Box & Muller 1958).  Everything is vectorised numpy on
uint64 (wrapping arithmetic), so the draws are identical on x86 and aarch64.

Workload shapes follow the paper's problem statement (Methods, "Training
Collocation Points" and "Solution Modeling"): 1D problems sample y >= 0 (the
profiles have a definite parity, so half of the line suffices), 2D problems
sample the quadrant y1 >= 0, y2 >= 0 above the wall y2 = 0, with extra
boundary points on the wall.  The exact regions and measures of the paper are
in its (unpublished) Supplementary Information; the recipes below are
synthetic stand-ins with the same structure (log-radial plus uniform mixes).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Equation identifiers shared with the C ABI (gn.h) and the oracle.
BURGERS, CCF, IPM, BOUSSINESQ = 0, 1, 2, 3
EQUATION_NAMES = {BURGERS: "burgers", CCF: "ccf", IPM: "ipm", BOUSSINESQ: "boussinesq"}
EQUATION_DIM = {BURGERS: 1, CCF: 1, IPM: 2, BOUSSINESQ: 2}
EQUATION_FIELDS = {BURGERS: 1, CCF: 1, IPM: 2, BOUSSINESQ: 3}


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n consecutive SplitMix64 outputs of stream `seed`, starting at draw `offset`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in (0, 1]: (top 53 bits + 1) * 2^-53."""
    z = splitmix64(seed, n, offset)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def signs(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Independent +-1 values (the top bit of each SplitMix64 draw), as doubles."""
    z = splitmix64(seed, n, offset)
    return np.where((z >> np.uint64(63)) == np.uint64(1), 1.0, -1.0)


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normal deviates by Box-Muller (one deviate per pair of uniforms)."""
    u = uniform(seed, 2 * n, 2 * offset)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------
# network parameters
# --------------------------------------------------------------------------

def param_count(widths: Sequence[int]) -> int:
    """Parameters of a dense MLP with the given layer widths (weights + biases)."""
    return int(sum(widths[i] * widths[i + 1] + widths[i + 1] for i in range(len(widths) - 1)))


def xavier_init(widths: Sequence[int], seed: int) -> np.ndarray:
    """Xavier-normal weights (std = sqrt(2/(fan_in+fan_out))), zero biases.

    Layout (the one the C ABI uses): for each layer l, W_l as an out x in
    row-major block, then b_l (out entries).
    """
    theta = np.zeros(param_count(widths))
    off = 0
    for l in range(len(widths) - 1):
        fi, fo = widths[l], widths[l + 1]
        std = math.sqrt(2.0 / (fi + fo))
        theta[off:off + fi * fo] = std * normal(seed * 1000003 + l, fi * fo)
        off += fi * fo + fo
    return theta


# --------------------------------------------------------------------------
# collocation sets
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    """One profile fit: equation, network shape, points and the lambda seed."""
    name: str
    equation: int
    widths: List[int]
    y: np.ndarray                 # (d, n_pts) interior collocation points
    y_bnd: np.ndarray             # (d, n_bnd) wall points (2D problems), may be empty
    lam: float
    theta: np.ndarray
    gamma: float = 1e-6
    hilbert_m: int = 1024         # CCF only: number of circle nodes of the Hilbert operator
    y_norm: tuple = (1.0, 0.0)
    c_norm: float = 1.0
    rho: Optional[np.ndarray] = None
    c_bnd: float = 1.0                   # weight of the wall loss
    c_norm_w: float = 1.0                # weight of the normalisation row
    y_inf: Optional[np.ndarray] = None   # (d, n_inf) decay points of the data loss, or None
    c_inf: float = 1.0
    norm_field: Optional[int] = None     # normalisation on another field / on d/dy1 (None: the
    norm_deriv: Optional[int] = None     # equation's own constraint)
    output_map: int = 0                  # last activation: 0 linear, 1 exp
    y_relu: Optional[np.ndarray] = None  # (d, n_relu) bound points of the data loss, or None
    c_relu: float = 1.0
    relu_bound: float = 0.0
    relu_sign: int = 1                   # +1 upper bound, -1 lower bound
    y_d1: Optional[np.ndarray] = None    # (d, n_d1) points of the d1 derivative loss, or None
    rho_d1: Optional[np.ndarray] = None
    c_d1: float = 1.0
    y_d2: Optional[np.ndarray] = None    # (d, n_d2) points of the d2 derivative loss, or None
    rho_d2: Optional[np.ndarray] = None
    c_d2: float = 1.0

    @property
    def d(self) -> int:
        return EQUATION_DIM[self.equation]

    @property
    def n_pts(self) -> int:
        return int(self.y.shape[1])

    @property
    def n_bnd(self) -> int:
        return int(self.y_bnd.shape[1]) if self.y_bnd.size else 0

    @property
    def n_params(self) -> int:
        return param_count(self.widths)


# Normalisation points (the paper fixes a point at a high-gradient region and
# a target value; the choice per equation is this project's reading).
NORM_POINT = {
    BURGERS: ((-2.0, 0.0), 1.0),      # U(-2) = 1: the lambda = 1/2, C = 1 closed form
    CCF: ((1.0, 0.0), 1.0),           # Theta(1) = 1
    IPM: ((1.0, 0.0), 1.0),           # P(1, 0) = 1
    BOUSSINESQ: ((0.0, 0.0), 1.0),    # d Omega / d y1 at the origin = 1
}


def _log_space(lo: float, hi: float, n: int) -> np.ndarray:
    if n == 1:
        return np.array([lo])
    return 10.0 ** np.linspace(math.log10(lo), math.log10(hi), n)


def points_1d(n_uniform: int, n_log: int, lo: float, hi: float, seed: int,
              uniform_lo: float = 0.0) -> np.ndarray:
    """Half uniform on [uniform_lo, hi], half log-spaced on [lo, hi]; shape (1, n)."""
    u = uniform_lo + (hi - uniform_lo) * uniform(seed, n_uniform)
    g = _log_space(lo, hi, n_log)
    return np.concatenate([g, u]).reshape(1, -1)


def points_2d_polar(n_r: int, n_a: int, r_lo: float, r_hi: float, seed: int,
                    random_radius: bool = False) -> np.ndarray:
    """Quadrant points: radii log-spaced (or 10^U) times uniform angles in [0, pi/2]."""
    if random_radius:
        n = n_r * n_a
        r = 10.0 ** (math.log10(r_lo) + (math.log10(r_hi) - math.log10(r_lo)) * uniform(seed, n))
        a = 0.5 * math.pi * uniform(seed + 7, n)
    else:
        r = np.repeat(_log_space(r_lo, r_hi, n_r), n_a)
        a = 0.5 * math.pi * uniform(seed, n_r * n_a)
    return np.stack([r * np.cos(a), r * np.sin(a)])


def wall_points(n: int, lo: float, hi: float, seed: int, random: bool = False) -> np.ndarray:
    if random:
        y1 = 10.0 ** (math.log10(lo) + (math.log10(hi) - math.log10(lo)) * uniform(seed, n))
    else:
        y1 = _log_space(lo, hi, n)
    return np.stack([y1, np.zeros(n)])


def _wl(name, eq, widths, y, y_bnd, lam, seed, gamma=1e-6, m=1024):
    (yn, cn) = NORM_POINT[eq]
    return Workload(name=name, equation=eq, widths=list(widths), y=np.ascontiguousarray(y),
                    y_bnd=np.ascontiguousarray(y_bnd), lam=float(lam),
                    theta=xavier_init(widths, seed), gamma=gamma, hilbert_m=m,
                    y_norm=yn, c_norm=cn)


def ccf_stable_1d(seed: int = 1) -> Workload:
    """CCF stable profile: MLP 1-32-32-1, 1024 points (512 uniform on [0, 1e3] + 512
    log-spaced on [1e-3, 1e3]), M = 1024 Hilbert nodes, damping 1e-6, lambda seed 1.0."""
    y = points_1d(512, 512, 1e-3, 1e3, seed)
    return _wl("ccf_stable_1d_mlp1x32x32x1_n1024", CCF, [1, 32, 32, 1], y, np.zeros((1, 0)), 1.0, seed)


def ccf_unstable_1d(seed: int = 2) -> Workload:
    """CCF 1st unstable profile: MLP 1-64-64-64-1, 16384 points (12288 log-spaced on
    [1e-3, 1e4] + 4096 uniform on [1e-3, 1e4]), lambda seed 0.6057 (the value the
    paper quotes for this profile)."""
    y = points_1d(4096, 12288, 1e-3, 1e4, seed, uniform_lo=1e-3)
    return _wl("ccf_unstable1_1d_mlp1x64x64x64x1_n16384", CCF, [1, 64, 64, 64, 1], y,
               np.zeros((1, 0)), 0.6057, seed)


def burgers_half_1d(seed: int = 6) -> Workload:
    """Burgers at lambda = 1/2 (the paper's worked example, whose smooth profile with U(-2) = 1
    is known in closed form): MLP 1-32-32-1, 1024 points (512 log-spaced on [1e-3, 1e3] + 512
    uniform on [1e-3, 1e3])."""
    y = points_1d(512, 512, 1e-3, 1e3, seed, uniform_lo=1e-3)
    return _wl("burgers_half_1d_mlp1x32x32x1_n1024", BURGERS, [1, 32, 32, 1], y, np.zeros((1, 0)), 0.5, seed)


def ipm_2d(seed: int = 4) -> Workload:
    """IPM with boundary: MLP 2-64x4-2, 256 log radii in [1e-3, 1e3] x 256 seeded angles,
    plus 4096 wall points; lambda seed 1/0.9723 (the paper's empirical law at n = 0)."""
    y = points_2d_polar(256, 256, 1e-3, 1e3, seed)
    yb = wall_points(4096, 1e-3, 1e3, seed)
    return _wl("ipm_2d_mlp2x64x4x2_n65536_b4096", IPM, [2, 64, 64, 64, 64, 2], y, yb,
               1.0 / 0.9723, seed)


def boussinesq_2d(seed: int = 5) -> Workload:
    """Boussinesq with boundary: MLP 2-128x4-3, 262144 points (r = 10^U(-3,3), angle
    U[0, pi/2]) plus 16384 wall points; lambda seed 1/1.0863 + 1 (paper's law at n = 0)."""
    y = points_2d_polar(512, 512, 1e-3, 1e3, seed, random_radius=True)
    yb = wall_points(16384, 1e-3, 1e3, seed, random=True)
    return _wl("boussinesq_2d_mlp2x128x4x3_n262144_b16384", BOUSSINESQ,
               [2, 128, 128, 128, 128, 3], y, yb, 1.0 / 1.0863 + 1.0, seed)


def batched_ccf_sweep(seed: int = 3, n_fits: int = 64) -> List[Workload]:
    """64 uneven CCF fits: width in {16,32,48,64}, hidden depth in {2,3},
    N ~ U{2048..16384}, lambda ~ U[0.5, 3]; points shaped like the 1st unstable set."""
    u = uniform(seed, 4 * n_fits)
    fits = []
    for f in range(n_fits):
        w = (16, 32, 48, 64)[min(3, int(u[4 * f] * 4))]
        depth = 2 if u[4 * f + 1] < 0.5 else 3
        n = 2048 + int(u[4 * f + 2] * (16384 - 2048 + 1))
        n = min(n, 16384)
        lam = 0.5 + 2.5 * u[4 * f + 3]
        n_uni = n // 4
        y = points_1d(n_uni, n - n_uni, 1e-3, 1e4, seed * 7919 + f, uniform_lo=1e-3)
        widths = [1] + [w] * depth + [1]
        fits.append(_wl(f"ccf_fit{f:02d}_w{w}_d{depth}_n{n}", CCF, widths, y, np.zeros((1, 0)),
                        lam, seed * 104729 + f))
    return fits


def small_case(equation: int, widths: Sequence[int], n_pts: int, n_bnd: int = 0,
               seed: int = 11, lam: Optional[float] = None, m: int = 64) -> Workload:
    """A small instance of any equation (for parity tests): points shaped like the
    full workloads but few of them, so the oracle finishes in seconds."""
    d = EQUATION_DIM[equation]
    if d == 1:
        n_log = n_pts // 2
        y = points_1d(n_pts - n_log, n_log, 1e-3, 1e3, seed, uniform_lo=1e-3)
        yb = np.zeros((1, 0))
    else:
        na = max(1, int(round(math.sqrt(n_pts))))
        nr = max(1, n_pts // na)
        y = points_2d_polar(nr, na, 1e-3, 1e2, seed)
        extra = n_pts - y.shape[1]
        if extra > 0:
            y = np.concatenate([y, points_2d_polar(extra, 1, 1e-2, 10.0, seed + 1)], axis=1)
        yb = wall_points(n_bnd, 1e-3, 1e2, seed + 2) if n_bnd else np.zeros((2, 0))
    if lam is None:
        lam = {BURGERS: 0.5, CCF: 0.6057, IPM: 1.0 / 0.9723, BOUSSINESQ: 1.0 / 1.0863 + 1.0}[equation]
    return _wl(f"small_{EQUATION_NAMES[equation]}", equation, widths, y, yb, lam, seed, m=m)


def weighted(w: Workload, seed: int = 31) -> Workload:
    """The same workload with non-unit loss weights: per-point weights rho ~ U[0.25, 4] and
    wall / normalisation weights 2.75 / 0.35 (the paper's d0 loss carries a weight per point;
    its data loss a coefficient per constraint)."""
    return dataclasses.replace(w, name=w.name + "_weighted", rho=0.25 + 3.75 * uniform(seed, w.n_pts),
                               c_bnd=2.75, c_norm_w=0.35)


def with_derivative_batches(w: Workload, n1: int, n2: int, seed: int = 41, c_d1: float = 0.3,
                            c_d2: float = 0.05) -> Workload:
    """The same workload with batches Y_1, Y_2 for the d1 and d2 derivative losses (the paper
    assigns each loss its own batch; its batches are in its Supplementary Information): seeded
    subsets of the collocation points with point weights rho ~ U[0.5, 2]."""
    n = w.n_pts
    pick1 = np.argsort(uniform(seed, n))[:n1]
    pick2 = np.argsort(uniform(seed + 1, n))[:n2]
    return dataclasses.replace(w, name=w.name + "_dloss", y_d1=np.ascontiguousarray(w.y[:, pick1]),
                               rho_d1=0.5 + 1.5 * uniform(seed + 2, n1), c_d1=c_d1,
                               y_d2=np.ascontiguousarray(w.y[:, pick2]), rho_d2=0.5 + 1.5 * uniform(seed + 3, n2),
                               c_d2=c_d2)


WORKLOADS = {
    "burgers_half": burgers_half_1d,
    "ccf_stable": ccf_stable_1d,
    "ccf_unstable1": ccf_unstable_1d,
    "ipm": ipm_2d,
    "boussinesq": boussinesq_2d,
}
