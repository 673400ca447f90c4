#!/usr/bin/env python
"""Benchmark: damped Gauss-Newton steps/s of a self-similar profile fit on GB300.

Workload (one GN step = the whole hot path): CCF 1st unstable profile, MLP
1-64-64-64-1 tanh (8513 parameters + lambda), 16384 collocation points
(12288 log-spaced on [1e-3, 1e4] + 4096 uniform), M = 1024 Hilbert nodes;
per step: jets -> residuals -> Jacobian rows (16385 x 8514), the Hilbert
contraction, Gram G = J~^T J~ and g = J~^T r~, damped FP64 Cholesky solve,
Armijo line search with residual-only evaluations, LM damping update.
Inputs are seeded and synthetic (the paper's collocation sets are defined in
its unpublished Supplementary Information).  J~ (1.1 GB) and G (0.58 GB)
exceed the 129 MB L2, so no explicit L2 flush is needed between steps.

Prints ONE JSON line (rank 0).  With --impl reference it times the CPU
oracle (numpy FP64, complex-step Jacobian) on a bounded sample of the same
step and extrapolates to one full step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one split Gram launch,
# ozaki_kernel<6,1,0> on the CCF 1st-unstable workload (2278 tiles, S = 6), from a single-pass
# ncu capture of `bench.py --eager --gram-split 1 --gram-tile 128 --steps 1 --warmup 1` (the eager
# path: ncu lists no kernels inside graphs with conditional nodes; split-K and tile width forced so
# that no tuning launch comes first) with the tiles in blocked order and the store loop free of
# FP64 conversions: 12.398 GB read + 0.306 GB written (18.18 + 0.31 GB in row order).  Valid only
# for that kernel build and workload; re-measure when either changes.
GRAM_TRAFFIC_BYTES_CCF_S6 = 12.398e9 + 0.306e9

METRIC = "gn_steps_per_s"
UNIT = "steps/s"
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (DFMA/DMMA) nominal; the probe measured 1.19 DFMA


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="split_all", choices=["fp64", "split", "split_all"])
    ap.add_argument("--slices", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the equal-residual and batched-sweep records of the default line")
    ap.add_argument("--extras-er-steps", type=int, default=50,
                    help="FP64 GN steps of the default line's equal-residual record (CCF stable profile)")
    ap.add_argument("--micro", default=None, choices=[None, "gram", "chol", "jacobian"],
                    help="time one kernel family alone instead of the GN step (not the bench contract line)")
    ap.add_argument("--width", type=int, default=None,
                    help="--micro: hidden width w of a 1-w-w-1 CCF net (gram: default 44; chol: default the "
                         "benchmark's 1-64-64-64-1 net)")
    ap.add_argument("--equal-residual", action="store_true",
                    help="FP64 path for --er-steps steps vs split path to the same max residual (own JSON line)")
    ap.add_argument("--er-steps", type=int, default=50,
                    help="--equal-residual: FP64 steps (the workload is --workload: ccf_unstable1, ccf_stable or ipm)")
    ap.add_argument("--ema-vs-exact", action="store_true",
                    help="head-to-head on the same kernels: exact-G damped GN vs the paper's EMA rank-1 "
                         "optimiser, loss against device time (own JSON line)")
    ap.add_argument("--ema-beta", type=float, default=0.95)
    ap.add_argument("--workload", default="ccf_unstable1",
                    choices=["ccf_unstable1", "ccf_stable", "ipm", "boussinesq", "batched"],
                    help="ccf_unstable1 is the headline line; the others print their own line")
    ap.add_argument("--streams", type=int, default=8, help="--workload batched: CUDA streams (host workers)")
    ap.add_argument("--multistage", action="store_true",
                    help="two-stage training (stage 2 learns the error of stage 1; own JSON line)")
    ap.add_argument("--stage-steps", type=int, nargs=2, default=[300, 300])
    ap.add_argument("--ms-workload", default="burgers_half", choices=["burgers_half", "ccf_stable"])
    ap.add_argument("--funnel", action="store_true",
                    help="funnel inference of lambda over a batch of fits at fixed lambda (own JSON line)")
    ap.add_argument("--funnel-fits", type=int, default=8)
    ap.add_argument("--funnel-workload", default="burgers_half",
                    choices=["ccf_stable", "ccf_unstable1", "ipm", "burgers_half"])
    ap.add_argument("--funnel-spread", type=float, default=0.2,
                    help="relative spread of the fits' lambda seeds around the workload's seed")
    ap.add_argument("--funnel-relax", type=int, default=1500,
                    help="GN steps at the seed lambda before the first r_hat (the fit relaxes first)")
    ap.add_argument("--funnel-iters", type=int, default=8)
    ap.add_argument("--funnel-steps", type=int, default=300)
    ap.add_argument("--funnel-radius", type=float, default=0.1)
    ap.add_argument("--funnel-dlam", type=float, default=0.01)
    ap.add_argument("--gram-split", type=int, default=0,
                    help="force the split Gram's split-K factor (0: autotuned per shape)")
    ap.add_argument("--gram-tile", type=int, default=0, choices=[0, 64, 128],
                    help="force the split Gram's output tile width (0: autotuned)")
    ap.add_argument("--pipeline", type=int, default=None,
                    help="tiles per Gram chunk of the pipelined graph step (-1: 7/8 of the SM count; "
                         "default: the library's, off: Gram then factorisation)")
    ap.add_argument("--eager", action="store_true",
                    help="step with gn_step (host decisions between launches) instead of the captured graphs; "
                         "--workload batched: one host worker thread per stream instead of the batched graph")
    ap.add_argument("--graph", action="store_true",
                    help="step through the captured CUDA graphs (gn_step_graph; batched: one graph launch per "
                         "batched step, gn_batch_graph_step)")
    ap.add_argument("--radii", type=int, default=None,
                    help="--micro jacobian on a 2D workload: radii x angles of a smaller point set (default: full)")
    return ap.parse_args()


def validation_grid_1d(n_log=60000, n_uni=40000):
    """Dense validation grid for the 1D max-d0 residual (the paper's grids are in its SI):
    log-spaced on [1e-4, 1e5] plus uniform on [0, 10] (uniform points start at 1e-4)."""
    import numpy as np
    g = np.concatenate([10.0 ** np.linspace(-4, 5, n_log), np.linspace(1e-4, 10.0, n_uni)])
    return g.reshape(1, -1)


def validation_grid_2d(n_r=512, n_a=256):
    """Dense 2D validation grid (the paper's grids are in its SI): radii log-spaced on
    [1e-4, 1e4] times angles uniform on [0, pi/2] (quadrant), 131072 points."""
    import numpy as np
    r = np.repeat(10.0 ** np.linspace(-4, 4, n_r), n_a)
    a = np.tile(np.linspace(0.0, 0.5 * np.pi, n_a), n_r)
    return np.stack([r * np.cos(a), r * np.sin(a)])


def equal_residual_record(workload, steps, precision="split_all", slices=6):
    """Split precision vs FP64 at equal residual.  The FP64 path takes `steps` GN steps from
    the seeded initialisation; the target is its final max d0 residual on the dense
    validation grid times 1.1.  The split path then steps from the same initialisation until
    it holds a state at least as converged as the FP64 path's final one: its own grid max d0
    residual at or below the target and its training loss at or below 1.1 x the FP64 path's
    final loss (the max d0 residual alone is not monotone early in a fit: a random-init
    network can touch a low maximum after one step while its loss is still high).  At most
    4 x steps.  The record gives both paths' device time (CUDA events around each gn_step;
    the grid evaluations run outside those events), or the residual gap if the split path
    never gets there."""
    import torch
    from paper_2509_14185_gb300 import gn, inputs
    w = inputs.WORKLOADS[workload]()
    grid = validation_grid_1d() if w.d == 1 else validation_grid_2d()
    val = gn.GNProblem(w.equation, w.widths, grid, y_norm=w.y_norm, c_norm=w.c_norm, hilbert_m=w.hilbert_m)

    def run(prec, max_steps, target=None, target_loss=None):
        prob = gn.GNProblem.from_workload(w, precision=prec, n_slices=slices)
        theta = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
        lam, gam = w.lam, w.gamma
        t_ms, hist = 0.0, []
        for k in range(max_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            rc, lam, gam, info = prob.gn_step(theta, lam, gam)
            e1.record()
            torch.cuda.synchronize()
            t_ms += e0.elapsed_time(e1)
            res = val.gn_max_residual(theta, lam)
            hist.append({"step": k + 1, "ms": t_ms, "max_res": res, "lambda": lam, "loss": info["loss_after"],
                         "rc": rc})
            if target is not None and res <= target and info["loss_after"] <= target_loss:
                break
        prob.close()
        return hist

    h64 = run(gn.GN_PREC_FP64, steps)
    target = h64[-1]["max_res"] * 1.1
    target_loss = h64[-1]["loss"] * 1.1
    prec = {"split": gn.GN_PREC_SPLIT_BF16, "split_all": gn.GN_PREC_SPLIT_ALL}.get(precision, gn.GN_PREC_SPLIT_ALL)
    hs = run(prec, 4 * steps, target, target_loss)
    reached = hs[-1]["max_res"] <= target and hs[-1]["loss"] <= target_loss
    val.close()
    return {"workload": w.name, "grid_points": int(grid.shape[1]),
            "target": "FP64 path's final max d0 residual on the validation grid x 1.1, with the training "
                      "loss at or below 1.1 x the FP64 path's final loss",
            "target_max_res": target, "target_loss": target_loss,
            "fp64": {"steps": len(h64), "device_s": h64[-1]["ms"] / 1e3, "max_res": h64[-1]["max_res"],
                     "loss": h64[-1]["loss"], "lambda": h64[-1]["lambda"]},
            "split": {"precision": precision, "slices": slices, "reached": reached, "steps": len(hs),
                      "device_s": hs[-1]["ms"] / 1e3, "max_res": hs[-1]["max_res"], "loss": hs[-1]["loss"],
                      "lambda": hs[-1]["lambda"]},
            "speedup_to_equal_residual": (h64[-1]["ms"] / hs[-1]["ms"]) if reached else None,
            "residual_gap": None if reached else {"max_res": min(h["max_res"] for h in hs) / target,
                                                  "loss": min(h["loss"] for h in hs) / target_loss},
            "fp64_curve": [(h["step"], h["max_res"], h["loss"]) for h in h64[::5]],
            "split_curve": [(h["step"], h["max_res"], h["loss"]) for h in hs[::5]]}


def equal_residual(args):
    """--equal-residual: the record of equal_residual_record for --workload, printed alone."""
    from paper_2509_14185_gb300 import build as B
    B.build()
    name = args.workload if args.workload in ("ccf_unstable1", "ccf_stable", "ipm") else "ccf_unstable1"
    out = dict({"mode": "equal_residual"}, **equal_residual_record(name, args.er_steps, args.precision, args.slices))
    print(json.dumps(out))
    return 0


def ema_vs_exact(args):
    """Exact-G damped GN (gn_step) against the paper's optimiser (gn_step_ema: EMA of rank-1
    curvature samples, closed-form learning rate and momentum) from the same initialisation,
    both in the chosen precision, for the same device-time budget: the exact path's --er-steps
    steps.  Reports the training loss against device time for both."""
    import numpy as np
    import torch
    from paper_2509_14185_gb300 import build as B
    B.build()
    from paper_2509_14185_gb300 import gn, inputs
    w = inputs.ccf_unstable_1d()
    prec = {"fp64": gn.GN_PREC_FP64, "split": gn.GN_PREC_SPLIT_BF16, "split_all": gn.GN_PREC_SPLIT_ALL}[args.precision]
    prob = gn.GNProblem.from_workload(w, precision=prec, n_slices=args.slices)
    Pp, R = prob.P + 1, prob.n_rows

    def curve_exact(n):
        th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
        lam, gam, t, out = w.lam, w.gamma, 0.0, []
        for k in range(n):
            rc, lam, gam, info = prob.gn_step(th, lam, gam)
            t += info["ms_phase"][6] * 1e-3
            out.append([k + 1, t, info["loss_after"]])
        return out, t

    def curve_ema(budget):
        th = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
        G = torch.zeros((Pp, Pp), dtype=torch.float64, device="cuda")
        v = torch.zeros(Pp, dtype=torch.float64, device="cuda")
        lam, gam, t, out, k = w.lam, w.gamma, 0.0, [], 0
        while t < budget and k < 100000:
            s = torch.tensor(inputs.signs(1234, R, R * k), dtype=torch.float64, device="cuda")
            rc, lam, gam, info = prob.gn_step_ema(th, lam, gam, G, v, s, args.ema_beta, k == 0)
            t += info["ms_phase"][6] * 1e-3
            k += 1
            out.append([k, t, info["loss_after"]])
        return out, t

    exact, budget = curve_exact(args.er_steps)
    ema, t_ema = curve_ema(budget)
    best_exact = min(c[2] for c in exact)
    best_ema = min(c[2] for c in ema)
    thin = lambda c: c[:: max(1, len(c) // 25)] + [c[-1]]
    print(json.dumps({"mode": "ema_vs_exact", "workload": w.name, "precision": args.precision,
                      "beta": args.ema_beta, "budget_device_s": budget,
                      "exact": {"steps": len(exact), "device_s": budget, "best_loss": best_exact,
                                "ms_per_step": 1e3 * budget / len(exact)},
                      "ema": {"steps": len(ema), "device_s": t_ema, "best_loss": best_ema,
                              "ms_per_step": 1e3 * t_ema / len(ema)},
                      "exact_curve": thin(exact), "ema_curve": thin(ema)}))
    prob.close()
    return 0


def micro_gram(args):
    """Split (or FP64) Gram product alone on a real CCF Jacobian: 16385 rows x P' columns,
    P' = w^2 + 4w + 2 (w = 44: 2114 columns, J = 277 MB, larger than L2).  Prints one
    JSON line with per-launch times from CUDA events (this is the small case used for
    detailed ncu captures of the Gram kernels)."""
    import numpy as np
    import torch
    from paper_2509_14185_gb300 import build as B
    B.build()
    from paper_2509_14185_gb300 import gn, inputs
    w = inputs.ccf_unstable_1d()
    width = args.width or 44
    w.widths = [1, width, width, 1]
    w.theta = inputs.xavier_init(w.widths, 17)
    prec = {"fp64": gn.GN_PREC_FP64, "split": gn.GN_PREC_SPLIT_BF16, "split_all": gn.GN_PREC_SPLIT_BF16}[args.precision]
    prob = gn.GNProblem.from_workload(w, precision=prec, n_slices=args.slices)
    Pp = prob.P + 1
    theta = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    J = torch.zeros((prob.n_rows, Pp), dtype=torch.float64, device="cuda")
    prob.gn_jacobian(theta, w.lam, J)
    G = torch.zeros((Pp, Pp), dtype=torch.float64, device="cuda")
    g = prob.new_vec(Pp)
    r = prob.new_vec(prob.n_rows)
    for _ in range(args.warmup):
        prob.gn_gram(J, prob.n_rows, r, G, g, precision=prec)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        prob.gn_gram(J, prob.n_rows, r, G, g, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    rows = prob.n_rows
    alg = rows * Pp * (Pp + 1.0)
    out = {"micro": "gram", "precision": args.precision, "slices": args.slices, "rows": rows, "cols": Pp,
           "ms_median": ms, "fp64_equivalent_tflops": alg / (ms * 1e-3) / 1e12}
    if prec != gn.GN_PREC_FP64:
        S = args.slices
        nt = -(-Pp // 128)
        kpad = -(-rows // 32) * 32
        executed = S * (S + 1) / 2 * (nt * (nt + 1) / 2) * 128 * 128 * kpad * 2.0
        out["tensor_tflops_incl_prepass"] = executed / (ms * 1e-3) / 1e12
    print(json.dumps(out))
    prob.close()
    return 0


def micro_jacobian(args):
    """The fused jet -> residual -> Jacobian-row kernel alone (gn_jacobian over all rows) and
    the residual-only pass of the line search (gn_residual), timed with CUDA events on the
    handle's stream.  Algorithmic bytes of the Jacobian pass: rows * P' * 8 written (the
    J~ rows; inputs and weights are O(N + P)).  For CCF the pass also holds the Hilbert node
    jets and the J_U contraction, so a Burgers problem on the same network and points (no
    nonlocal term) is timed beside it: that line is the jet kernel alone.  Prints one JSON
    line (not the bench contract line); with --steps 1 --warmup 0 it is the small case of
    the jet-kernel ncu captures."""
    import torch
    from paper_2509_14185_gb300 import build as B
    B.build()
    from paper_2509_14185_gb300 import gn, inputs
    w = inputs.WORKLOADS[args.workload]()
    if args.radii and w.d == 2:
        seed = inputs.WORKLOADS[args.workload].__defaults__[0]
        w.y = inputs.points_2d_polar(args.radii, args.radii, 1e-3, 1e3, seed)
        w.y_bnd = inputs.wall_points(max(1, args.radii * args.radii // 16), 1e-3, 1e3, seed)
        w.name = w.name + f"_reduced_{args.radii}x{args.radii}"
    hbm, hsrc = measured_peak("hbm_gbs", 6800.0)
    cases = [(w.name, w.equation)]
    if w.equation == inputs.CCF:
        cases.append((w.name.replace("ccf", "burgers_same_net_and_points"), inputs.BURGERS))
    prec = {"fp64": gn.GN_PREC_FP64, "split": gn.GN_PREC_SPLIT_BF16, "split_all": gn.GN_PREC_SPLIT_ALL}[args.precision]
    out = {"micro": "jacobian", "hbm_peak_gbs": hbm, "peak_source": hsrc, "precision": args.precision, "cases": []}
    for name, eq in cases:
        prob = gn.GNProblem(eq, w.widths, w.y, w.y_bnd if w.y_bnd.size else None, w.rho, y_norm=w.y_norm,
                            c_norm=w.c_norm, hilbert_m=w.hilbert_m, precision=prec, n_slices=args.slices)
        Pp = prob.P + 1
        theta = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
        J = torch.empty((prob.n_rows, Pp), dtype=torch.float64, device="cuda")
        r = prob.new_vec(prob.n_rows)
        stream = torch.cuda.current_stream()

        def timed(fn):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            ts = []
            for _ in range(max(1, args.steps)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return statistics.median(ts)

        ms_j = timed(lambda: prob.gn_jacobian(theta, w.lam, J))
        ms_r = timed(lambda: prob.gn_residual(theta, w.lam, r, want_loss=False))
        jbytes = prob.n_rows * Pp * 8.0
        gbs = jbytes / (ms_j * 1e-3) / 1e9
        out["cases"].append({"case": name, "rows": prob.n_rows, "cols": Pp, "n_pts": prob.n_pts,
                             "jacobian_ms": ms_j, "jacobian_bytes_written": jbytes, "jacobian_gbs": gbs,
                             "jacobian_frac_hbm": gbs / hbm, "residual_ms": ms_r,
                             "residual_points_per_s": prob.n_pts / (ms_r * 1e-3),
                             "includes_hilbert": eq == inputs.CCF})
        del J
        prob.close()
    print(json.dumps(out))
    return 0


def run_multistage(args):
    """Two-stage training (Methods, "Multi-stage Training") on the GPU.  Stage 1 trains the
    workload's network at its fixed lambda (Burgers: the admissible lambda = 1/2) for
    --stage-steps[0] damped GN steps (captured graphs); eps = its max residual on the
    collocation points.  Stage 2 freezes it and trains a second network on the stage-2
    problem (fields Phi_1 + eps Phi_2, rows / eps) for --stage-steps[1] steps, in two
    variants: a tanh MLP of the stage-1 shape, and the paper's Fourier-feature network whose
    B ~ N(0, sigma^2) has sigma = 2 pi f_d, f_d the dominant frequency of the stage-1
    residual as a function of the network input q (FFT on a uniform q grid).  Reports the max
    d0 residual on a dense grid inside the training range after each stage, and for Burgers
    the max error against the closed-form profile (U^3 + U + y = 0)."""
    import numpy as np
    import torch
    from paper_2509_14185_gb300 import build as B
    B.build()
    from paper_2509_14185_gb300 import gn, inputs
    w = inputs.WORKLOADS[args.ms_workload]()
    prec = {"fp64": gn.GN_PREC_FP64, "split": gn.GN_PREC_SPLIT_BF16, "split_all": gn.GN_PREC_SPLIT_ALL}[args.precision]
    grid = np.concatenate([10.0 ** np.linspace(-3, 3, 60000), np.linspace(1e-3, 10.0, 40000)]).reshape(1, -1)

    def make(widths, fourier=None, pts=None):
        return gn.GNProblem(w.equation, widths, w.y if pts is None else pts, y_norm=w.y_norm, c_norm=w.c_norm,
                            hilbert_m=w.hilbert_m, precision=prec, n_slices=args.slices, fourier_B=fourier)

    def train(prob, theta, lam, n):
        gam, hist = w.gamma, []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(n):
            rc, lam2, gam, info = prob.gn_step_graph(theta, lam, gam)
            hist.append(info["loss_after"])
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3, hist

    lam = w.lam
    p1 = make(w.widths)
    p1.gn_set_lambda_trainable(False)
    th1 = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    s1, h1 = train(p1, th1, lam, args.stage_steps[0])
    eps = p1.gn_max_residual(th1, lam)
    v1 = make(w.widths, pts=grid)
    res1 = v1.gn_max_residual(th1, lam)

    def exact_err(fields):
        if w.equation != inputs.BURGERS:
            return None
        yv = grid[0]
        sq = np.sqrt(yv * yv / 4.0 + 1.0 / 27.0)
        U = np.cbrt(-yv / 2.0 + sq) + np.cbrt(-yv / 2.0 - sq)
        return float(np.max(np.abs(fields - U)))

    U1 = p1.gn_field_jets(th1, lam, grid).cpu().numpy()[:, 0]
    out = {"mode": "multistage", "workload": w.name, "precision": args.precision, "lambda": lam,
           "grid": "1e5 points inside the training range", "eps": eps,
           "stage1": {"steps": len(h1), "device_s": s1, "loss": h1[-1], "max_res_grid": res1,
                      "max_err_exact": exact_err(U1)}}

    # dominant frequency of the stage-1 residual in the network input q = (1 + y^2)^(-1/(2(1+lam)))
    qg = np.linspace((1.0 + 1e6) ** (-0.5 / (1.0 + lam)), (1.0 + 1e-6) ** (-0.5 / (1.0 + lam)), 4096)
    yq = np.sqrt(np.maximum(qg ** (-2.0 * (1.0 + lam)) - 1.0, 1e-12)).reshape(1, -1)
    vq = make(w.widths, pts=yq)
    r, _ = vq.residual(th1, lam)
    Rq = r.cpu().numpy()[:-1] / np.sqrt(2.0 / yq.shape[1])
    spec = np.abs(np.fft.rfft(Rq - Rq.mean()))
    kd = int(np.argmax(spec[1:]) + 1)
    f_d = kd / (qg[-1] - qg[0])
    sigma = 2.0 * np.pi * f_d
    out["fourier_sigma"] = sigma
    out["residual_dominant_frequency"] = f_d

    m, mf = 16, 16
    variants = [("tanh", list(w.widths), None,
                 inputs.xavier_init(w.widths, 777)),
                ("fourier", [1, m, 2 * mf, w.widths[-2], 1], sigma * inputs.normal(778, mf * m).reshape(mf, m),
                 None)]
    for name, widths2, Bm, th_init in variants:
        if th_init is None:
            P2 = (widths2[0] * m + m) + (2 * mf * widths2[3] + widths2[3]) + (widths2[3] + 1)
            th_init = 0.3 * inputs.normal(779, P2)
        p2 = make(widths2, Bm)
        p2.gn_set_stage1(w.widths, th1, lam, eps)
        th2 = torch.tensor(th_init, dtype=torch.float64, device="cuda")
        s2, h2 = train(p2, th2, lam, args.stage_steps[1])
        v2 = make(widths2, Bm, pts=grid)
        v2.gn_set_stage1(w.widths, th1, lam, eps)
        res2 = v2.gn_max_residual(th2, lam)
        U2 = v2.gn_field_jets(th2, lam, grid).cpu().numpy()[:, 0]
        out["stage2_" + name] = {"mlp": widths2, "steps": len(h2), "device_s": s2, "loss": h2[-1],
                                 "max_res_grid": res2, "gain_max_res": res1 / res2 if res2 > 0 else None,
                                 "max_err_exact": exact_err(U1 + eps * U2),
                                 "loss_curve": h2[:: max(1, len(h2) // 6)]}
        for q in (p2, v2):
            q.close()
    print(json.dumps(out))
    for q in (p1, v1, vq):
        q.close()
    return 0


def run_funnel(args):
    """Funnel inference of lambda (Methods, "Identifying Admissible lambda Values", item 3)
    over a batch of fits: --funnel-fits copies of the workload with different seeded point
    sets and initialisations and lambda seeds spread evenly over +-(--funnel-spread)/2 of the
    workload's seed (default: Burgers around its admissible lambda = 1/2), each
    held at a fixed lambda (gn_set_lambda_trainable(0)) and trained --funnel-steps damped GN
    steps per iteration (one batched CUDA-graph launch per step); then r_hat(lambda), the
    signed residual of largest magnitude within --funnel-radius of the origin, is read for
    every fit and each fit's lambda moves by the secant update (gn_funnel_next).  Prints one
    JSON line with the lambda and r_hat histories and the device time per funnel iteration."""
    import torch
    from paper_2509_14185_gb300 import build as B
    B.build()
    from paper_2509_14185_gb300 import gn, inputs
    make = inputs.WORKLOADS[args.funnel_workload]
    seed0 = make.__defaults__[0]
    fits = []
    for f in range(args.funnel_fits):
        w = make(seed=seed0 + 100 + f)
        w.lam = w.lam * (1.0 + args.funnel_spread * (f / max(1, args.funnel_fits - 1) - 0.5))
        fits.append(w)
    prec = {"fp64": gn.GN_PREC_FP64, "split": gn.GN_PREC_SPLIT_BF16, "split_all": gn.GN_PREC_SPLIT_ALL}[args.precision]
    batch = gn.GNBatch(fits, n_streams=min(8, len(fits)), precision=prec, n_slices=args.slices)
    batch.gn_set_lambda_trainable(False)
    thetas = [torch.tensor(w.theta, dtype=torch.float64, device="cuda") for w in fits]
    batch.gn_batch_capture_graph(thetas)
    lams = [w.lam for w in fits]
    gams = [w.gamma for w in fits]
    hist_l = [[l] for l in lams]
    hist_r = [[] for _ in fits]
    iter_ms, losses = [], []
    for _ in range(args.funnel_relax):      # relax at the seed lambda first
        lams2, gams, infos, st = batch.gn_batch_graph_step(lams, gams)
    for it in range(args.funnel_iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.funnel_steps):
            lams2, gams, infos, st = batch.gn_batch_graph_step(lams, gams)
            assert lams2 == lams          # lambda is held fixed during the relaxation
        r = [batch.gn_signed_max_residual(f, thetas[f], lams[f], args.funnel_radius)[0] for f in range(len(fits))]
        e1.record()
        torch.cuda.synchronize()
        iter_ms.append(e0.elapsed_time(e1))
        losses.append(statistics.median(i["loss_after"] for i in infos))
        for f in range(len(fits)):
            hist_r[f].append(r[f])
            try:
                nxt = gn.gn_funnel_next(hist_l[f], hist_r[f], args.funnel_dlam)
            except gn.GNError:
                nxt = lams[f]
            lams[f] = nxt
            hist_l[f].append(nxt)
    batch.close()
    final = [h[-1] for h in hist_l]
    print(json.dumps({"mode": "funnel_inference", "workload": fits[0].name, "fits": len(fits),
                      "precision": args.precision, "relax_steps": args.funnel_relax,
                      "steps_per_iteration": args.funnel_steps,
                      "radius": args.funnel_radius, "dlambda": args.funnel_dlam,
                      "ms_per_iteration": statistics.median(iter_ms),
                      "fit_steps_per_s": len(fits) * args.funnel_steps / (statistics.median(iter_ms) * 1e-3),
                      "median_loss_per_iteration": losses,
                      "lambda_final": {"median": statistics.median(final), "min": min(final), "max": max(final)},
                      "lambda_history": hist_l[:: max(1, len(hist_l) // 4)],
                      "r_hat_history": hist_r[:: max(1, len(hist_r) // 4)]}))
    return 0


def replica_workload(name, rank):
    """Replicas: rank k fits its own profile, seeded with the workload's default seed + k
    (no data-path collective; the units of all ranks add up)."""
    from paper_2509_14185_gb300 import inputs
    if name == "batched":
        return inputs.batched_ccf_sweep(seed=3 + rank)
    make = inputs.WORKLOADS[name]
    return make(seed=make.__defaults__[0] + rank)


def max_over_ranks(x, device):
    """The slowest rank's time (the bench reports whole-job throughput over it)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_step_estimate(budget_cols=12, chol_n=512, gram_cols=512, workload="ccf_unstable1", _cache={}):
    """Time the oracle's pieces of one GN step on a bounded sample and extrapolate.

    Sample: complex-step Jacobian columns (`budget_cols` of the 8514, each a full
    residual evaluation over all 16384 points and the Hilbert nodes), the Gram
    product on a `gram_cols`-column slice of J~, the textbook Cholesky on a
    chol_n x chol_n SPD matrix, and one residual evaluation for the line search.
    Full step = P' * t_col + t_gram * (P'(P'+1)/(c(c+1))) + t_chol * (P'/n)^3 + 2 t_res.
    """
    import warnings

    import numpy as np

    from oracle import gn as ogn
    from oracle import problems as Pb
    from paper_2509_14185_gb300 import inputs as I

    warnings.filterwarnings("ignore", category=RuntimeWarning)
    if workload not in _cache:
        w = I.WORKLOADS[workload]()
        p = Pb.Problem(w.equation, w.widths, w.y, w.y_bnd if w.y_bnd.size else None, w.rho, y_norm=w.y_norm,
                       c_norm=w.c_norm, hilbert_m=w.hilbert_m)
        p.rows(w.theta, w.lam)   # first call pays numpy/BLAS start-up; not timed
        _cache[workload] = (p, w)
    p, w = _cache[workload]
    Pp = p.P + 1
    t0 = time.perf_counter()
    r = p.rows(w.theta, w.lam)
    t_res = time.perf_counter() - t0
    cols = np.linspace(0, p.P, budget_cols).astype(int)
    t0 = time.perf_counter()
    Jc = ogn.jacobian(p, w.theta, w.lam, cols)
    t_col = (time.perf_counter() - t0) / budget_cols
    rng = np.random.default_rng(0)
    Js = rng.standard_normal((p.n_rows, gram_cols))
    t0 = time.perf_counter()
    _ = Js.T @ Js
    _ = Js.T @ r
    t_gram = (time.perf_counter() - t0) * (Pp * (Pp + 1.0)) / (gram_cols * (gram_cols + 1.0))
    B = rng.standard_normal((chol_n + 8, chol_n))
    A = B.T @ B + np.eye(chol_n)
    t0 = time.perf_counter()
    L, ok = ogn.cholesky(A)
    ogn.cholesky_solve(L, np.ones(chol_n))
    t_chol = (time.perf_counter() - t0) * (Pp / chol_n) ** 3
    total = Pp * t_col + t_gram + t_chol + 2 * t_res
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    sample = (f"oracle (numpy FP64, complex-step J) on the same workload ({w.name}): {budget_cols} of {Pp} "
              f"Jacobian columns over all {p.n_rows} rows, Gram on a {gram_cols}-column slice, textbook Cholesky "
              f"n={chol_n}, 1 residual pass; extrapolated to one full step ({total:.1f} s)")
    return {"value": 1.0 / total, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "seconds_per_step_extrapolated": total, "parts_s": {"jacobian": Pp * t_col, "gram": t_gram,
                                                                  "cholesky": t_chol, "residuals": 2 * t_res}}


def micro_chol(args):
    """Damped Cholesky solve alone on the benchmark's own Gram matrix (CCF 1st unstable,
    P' = 8514): G from the GPU Jacobian, then gn_damped_solve timed with CUDA events.
    Prints one JSON line (not the bench contract line)."""
    import torch
    from paper_2509_14185_gb300 import build as B
    B.build()
    from paper_2509_14185_gb300 import gn, inputs
    w = inputs.ccf_unstable_1d()
    if args.width:
        w.widths = [1, args.width, args.width, 1]
        w.theta = inputs.xavier_init(w.widths, 17)
    prec = {"fp64": gn.GN_PREC_FP64, "split": gn.GN_PREC_SPLIT_BF16, "split_all": gn.GN_PREC_SPLIT_ALL}[args.precision]
    prob = gn.GNProblem.from_workload(w, precision=prec, n_slices=args.slices)
    Pp = prob.P + 1
    theta = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    J = torch.zeros((prob.n_rows, Pp), dtype=torch.float64, device="cuda")
    prob.gn_jacobian(theta, w.lam, J)
    r, _ = prob.residual(theta, w.lam)
    G = torch.zeros((Pp, Pp), dtype=torch.float64, device="cuda")
    g = prob.new_vec(Pp)
    prob.gn_gram(J, prob.n_rows, r, G, g, precision=gn.GN_PREC_FP64)
    G = torch.tril(G) + torch.tril(G, -1).T
    del J
    delta = prob.new_vec(Pp)
    for _ in range(args.warmup):
        prob.gn_damped_solve(G, g, w.gamma, delta)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rc, gam, retries = prob.gn_damped_solve(G, g, w.gamma, delta)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    A = G + gam * torch.eye(Pp, dtype=torch.float64, device="cuda")
    res = float((A @ delta - g).abs().max() / (A.abs().max() * delta.abs().max()))
    print(json.dumps({"micro": "chol", "precision": args.precision, "n": Pp, "ms_median": statistics.median(times),
                      "ms_min": min(times), "rc": rc, "retries": retries, "backward_error": res,
                      "diag_arith": "double-float"}))
    prob.close()
    return 0


def step_iqr(per):
    """Interquartile range of per-step times (0 for fewer than four steps)."""
    if len(per) < 4:
        return 0.0
    q = statistics.quantiles(per, n=4)
    return q[2] - q[0]


def measured_peak(key, default):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))[key]), "measured (MEASURED_PEAKS.json " + key + ")"
    except Exception:
        return default, "fallback"


def gram_executed_flops(rows, Pp, S):
    """Tensor-pipe FLOP of one split Gram launch: S(S+1)/2 slice pairs over the 128 x 128
    lower-triangular tiles of G and the 128-padded K (the Ozaki overhead included)."""
    nt = -(-Pp // 128)
    kpad = -(-rows // 128) * 128
    return S * (S + 1) / 2 * (nt * (nt + 1) / 2) * 128 * 128 * kpad * 2.0


def kernel_report(prob, args, phases, pipe_tiles=0):
    """Roofline entries of the step's dense phases (algorithmic FLOP / measured phase time).

    Gram: rows * P'(P'+1) FLOP (symmetric half).  FP64 path: DFMA pipe against the
    nominal FP64 peak.  Split paths: the tensor-pipe utilisation of the slice
    products actually executed (S(S+1)/2 pairs over the 128 x 128 lower-triangular
    tiles and the 128-padded K) against the measured sustained BF16 peak, plus the
    FP64-equivalent TFLOP/s.  Cholesky: P'^3/3 FLOP; on the FP64 path against the
    DFMA pipe, on the SPLIT_ALL path reported as FP64-equivalent TFLOP/s only (its
    time is shared between the FP64 diagonal factors, which are latency-bound on one
    SM each, and the tensor-core panel solves and trailing updates)."""
    Pp = prob.P + 1
    rows = prob.n_rows
    gram_ms, chol_ms = phases[1], phases[3]
    gram_flops = rows * Pp * (Pp + 1.0)
    fp64_src = "GB300 nominal FP64 1.25 TFLOP/s (DFMA probe on this pool: 1.19)"
    out = {}
    if args.precision == "fp64":
        a = gram_flops / (gram_ms * 1e-3) / 1e12
        out["gram"] = {"bound": "alu", "achieved": a, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                       "frac": a / FP64_NOMINAL_TFLOPS, "traffic": None, "ms": gram_ms,
                       "kernel": "dgemm_kernel<0,0> (FP64 Gram G = J~^T J~, DFMA pipe)",
                       "peak_source": fp64_src, "algorithmic_flops_per_launch": gram_flops}
    else:
        S = args.slices
        pk, src = measured_peak("bf16_tflops_sustained", 1700.0)
        executed = gram_executed_flops(rows, Pp, S)
        tens = executed / (gram_ms * 1e-3) / 1e12
        alg = gram_flops / (gram_ms * 1e-3) / 1e12
        # DRAM bytes of the whole-triangle launch from one ncu capture; the pipelined step's
        # chunk launches run inside a graph with conditional nodes, where ncu lists no kernels
        traffic = (GRAM_TRAFFIC_BYTES_CCF_S6 if (S == 6 and getattr(args, "workload", "") == "ccf_unstable1"
                                                 and not pipe_tiles) else None)
        out["gram"] = {"bound": "tensor", "achieved": alg, "peak": pk, "unit": "TFLOP/s", "frac": alg / pk,
                       "achieved_units": "algorithmic FLOP rows * P'(P'+1) (the symmetric half of J~^T J~, "
                                         "FP64-equivalent) per launch / the Gram phase time; the split "
                                         "path's extra slice products count as overhead",
                       "tensor_pipe": {"executed_tflops": tens, "frac": tens / pk,
                                       "executed_flops_per_launch": executed,
                                       "note": f"{S * (S + 1) // 2} BF16 slice-pair products per FP64-accurate "
                                               "entry, over the 128 x 128 lower tiles and 128-padded K"},
                       "traffic": traffic, "traffic_unit": "bytes per launch" if traffic else None, "ms": gram_ms,
                       "kernel": f"ozaki_kernel<{S},1,0> (split Gram: BF16 slice products on tcgen05, TMEM "
                                 "accumulators; the slicing pre-pass is inside the timed phase)",
                       "peak_source": src + ", sustained: the kernel runs inside a long step",
                       **({"pipelined": f"column-major chunks of <= {pipe_tiles} tiles on the lowest-priority "
                                        "stream beside the factorisation; ms is the Gram's wall time (slicing "
                                        "to its last chunk) while it shares the SMs with the factorisation"}
                          if pipe_tiles else {}),
                       "fp64_equivalent_tflops": alg,
                       "algorithmic_flops_per_launch": gram_flops}
    cf = Pp ** 3 / 3.0
    c = cf / (chol_ms * 1e-3) / 1e12
    if args.precision == "split_all":
        out["cholesky"] = {"bound": "mixed", "fp64_equivalent_tflops": c, "ms": chol_ms,
                           "kernel": "potrf_blk_kernel (blocked double-float 64 x 64 diagonal factor and "
                                     "inverse, one CTA) + panel_df_kernel (double-float panel solve writing the "
                                     f"split operand) + ozaki_kernel<{args.slices},0> (in-strip updates) + "
                                     f"ozaki_kernel<{args.slices},1> (K = 256 bulk updates, double-FP32 "
                                     "accumulation, overlapped with the next strip on a second stream); the phase "
                                     "includes the backward triangular solve",
                           "algorithmic_flops_per_launch": cf}
    else:
        out["cholesky"] = {"bound": "alu", "achieved": c, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                           "frac": c / FP64_NOMINAL_TFLOPS, "traffic": None, "ms": chol_ms,
                           "kernel": "potrf_inv_kernel<Arith64> + panel_solve_kernel + dgemm_kernel<1,1> "
                                     "(blocked FP64 Cholesky, DFMA pipe)",
                           "peak_source": fp64_src, "algorithmic_flops_per_launch": cf}
    out["jacobian"] = {"ms": phases[0], "note": "jets + residual + J rows (FP64 pipe); CCF adds the Hilbert "
                                                "contraction (FP64 DGEMM, or split on tcgen05 under SPLIT_ALL)"}
    return out


def mlp_name(widths):
    inner = widths[1:-1]
    if len(set(inner)) == 1 and len(inner) > 1:
        return f"{widths[0]}-{inner[0]}x{len(inner)}-{widths[-1]} tanh"
    return "-".join(str(v) for v in widths) + " tanh"


def workload_config(w, precision, slices):
    from paper_2509_14185_gb300 import inputs as I
    rows = w.n_pts * I.EQUATION_FIELDS[w.equation] + w.n_bnd + 1
    J_gb = rows * (w.n_params + 1) * 8 / 1e9
    return {"workload": w.name, "equation": I.EQUATION_NAMES[w.equation],
            "mlp": mlp_name(w.widths), "params": int(w.n_params) + 1, "n_pts": int(w.n_pts),
            "n_bnd": int(w.n_bnd), "rows": int(rows),
            "hilbert_nodes": int(w.hilbert_m) if w.equation == I.CCF else None,
            "gram_precision": precision if precision == "fp64" else f"split_bf16_s{slices}",
            "l2": f"working set (J~ {J_gb:.2f} GB) larger than the 129 MB L2; no flush needed"
                  if J_gb > 0.2 else "small working set: fits in L2 between steps",
            "parallelism": "replicas"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2509_14185_gb300 import inputs as I
    w = I.ccf_unstable_1d()
    times = []
    last = None
    for i in range(args.warmup + args.steps):
        est = oracle_step_estimate(budget_cols=4, chol_n=384, gram_cols=256)
        last = est
        if i >= args.warmup:
            times.append(est["seconds_per_step_extrapolated"])
    sec = statistics.mean(times)
    value = 1.0 / sec
    cb = dict(last)
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, "fp64", 0),
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_batched(args):
    """--workload batched: the batched sweep's own JSON line (see batched_record)."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2509_14185_gb300 import build as B
    B.build()
    line = batched_record(args, args.steps, args.warmup, rank, world)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def batched_record(args, steps, warmup, rank=0, world=1):
    """64 uneven CCF fits (widths 16..64, depth 2-3, 2048..16384 points, lambda ~ U[0.5, 3])
    stepped together: by default as one CUDA graph launch per batched step (every fit a
    branch; --eager: gn_batch_step on `--streams` CUDA streams).  value = fit-steps/s
    (64 x steps / time).  Each batched step returns only after its work is done, so the span
    between two events on an otherwise idle stream, recorded before and after the K batched
    steps, is the device-clock time of the whole batch."""
    import torch
    from paper_2509_14185_gb300 import gn, inputs
    if world > 1:
        import torch.distributed as dist
    fits = replica_workload("batched", rank)
    prec = {"fp64": gn.GN_PREC_FP64, "split": gn.GN_PREC_SPLIT_BF16, "split_all": gn.GN_PREC_SPLIT_ALL}[args.precision]
    batch = gn.GNBatch(fits, n_streams=args.streams, precision=prec, n_slices=args.slices)
    if args.gram_split:
        for f in range(len(fits)):
            gn.lib().gn_set_gram_split(batch.handle(f), int(args.gram_split))
    thetas = [torch.tensor(w.theta, dtype=torch.float64, device="cuda") for w in fits]
    lams = [w.lam for w in fits]
    gams = [w.gamma for w in fits]
    if args.graph or not args.eager:
        batch.gn_batch_capture_graph(thetas)
        step = lambda l, g: batch.gn_batch_graph_step(l, g)
    else:
        step = lambda l, g: batch.gn_batch_step(thetas, l, g)
    for _ in range(warmup):
        lams, gams, infos, st = step(lams, gams)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    L = gn.lib()
    launches0 = L.gn_kernel_launches()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    statuses = []
    ev0.record(stream)
    for _ in range(steps):
        lams, gams, infos, st = step(lams, gams)
        statuses.append(st)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = L.gn_kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1) / steps
    if world > 1:
        ms = max_over_ranks(ms, "cuda")
        dist.barrier()
    n = len(fits)
    value = world * n * 1000.0 / ms
    rows = [w.n_pts + 1 for w in fits]
    # the Gram tile shape and split-K factor the autotuner chose for each fit's shape
    import ctypes
    tiles, splits = {}, {}
    for f in range(n):
        t, k = ctypes.c_int(0), ctypes.c_int(0)
        hf = batch.handle(f)
        gn.lib().gn_gram_tile_choice(hf, rows[f], ctypes.byref(t))
        gn.lib().gn_gram_split_choice(hf, rows[f], ctypes.byref(k))
        tiles[t.value] = tiles.get(t.value, 0) + 1
        splits[k.value] = splits.get(k.value, 0) + 1
    Pps = [w.n_params + 1 for w in fits]
    gram_flops = sum(r * p * (p + 1.0) for r, p in zip(rows, Pps))
    chol_flops = sum(p ** 3 / 3.0 for p in Pps)
    line = None
    if rank == 0:
        kern = {"batched_step": {"ms": ms, "fp64_equivalent_gram_tflops": gram_flops / (ms * 1e-3) / 1e12,
                                 "fp64_equivalent_cholesky_tflops_if_alone": chol_flops / (ms * 1e-3) / 1e12}}
        roof = None
        if prec != gn.GN_PREC_FP64:
            pk, src = measured_peak("bf16_tflops_sustained", 1700.0)
            ex = sum(gram_executed_flops(r, p, args.slices) for r, p in zip(rows, Pps))
            a = ex / (ms * 1e-3) / 1e12
            roof = {"bound": "tensor", "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk,
                    "traffic": None, "kernel": f"ozaki_kernel<{args.slices},1> Gram launches of all fits",
                    "note": "executed Gram slice-product FLOP of all fits / whole batched step time "
                            "(a lower bound on the Gram kernels' own rate)", "peak_source": src}
        line = {"metric": "gn_fit_steps_per_s", "value": value, "unit": "fit-steps/s", "n_gpus": world,
                "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"batched_ccf_sweep_{n}_fits", "fits": n,
                           "gram_split": args.gram_split or "autotuned",
                           "gram_choices": {"tile_width_fits": {str(k): v for k, v in sorted(tiles.items())},
                                            "split_k_fits": {str(k): v for k, v in sorted(splits.items())}},
                           "launch": "one CUDA graph launch per batched step (every fit a branch)"
                           if (args.graph or not args.eager)
                           else f"{args.streams} streams, one host worker thread each",
                           "params_range": [min(Pps), max(Pps)], "n_pts_range": [min(rows) - 1, max(rows) - 1],
                           "gram_precision": args.precision if args.precision == "fp64"
                           else f"split_bf16_s{args.slices}",
                           "l2": "working set (all fits' J~, several GB) larger than L2; no flush needed",
                           "parallelism": "replicas"},
                "roofline": roof, "kernels": kern, "cpu_baseline": None, "e2e": None, "clocks": clocks,
                "gpu_launches": int(launches),
                "final": {"loss_mean": statistics.mean(i["loss_after"] for i in infos),
                          "warnings": sum(1 for st in statuses for x in st if x != 0)}}
    batch.close()
    return line


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.micro == "gram":
        return micro_gram(args)
    if args.micro == "chol":
        return micro_chol(args)
    if args.micro == "jacobian":
        return micro_jacobian(args)
    if args.equal_residual:
        return equal_residual(args)
    if args.funnel:
        return run_funnel(args)
    if args.multistage:
        return run_multistage(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.ema_vs_exact:
        return ema_vs_exact(args)
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2509_14185_gb300 import build as B
    B.build()
    from paper_2509_14185_gb300 import gn, inputs

    # replicas: every rank fits its own seeded profile (no data-path collective)
    w = replica_workload(args.workload, rank)
    prec = {"fp64": gn.GN_PREC_FP64, "split": gn.GN_PREC_SPLIT_BF16, "split_all": gn.GN_PREC_SPLIT_ALL}[args.precision]
    prob = gn.GNProblem.from_workload(w, precision=prec, n_slices=args.slices)
    if args.pipeline is not None:
        prob.gn_set_pipeline(args.pipeline)
    if args.gram_split:
        prob.gn_set_gram_split(args.gram_split)
    if args.gram_tile:
        prob.gn_set_gram_tile(args.gram_tile)
    stream = torch.cuda.current_stream()
    theta = torch.tensor(w.theta, dtype=torch.float64, device="cuda")
    lam, gam = w.lam, w.gamma
    use_graph = args.graph or not args.eager
    gn_step = prob.gn_step_graph if use_graph else prob.gn_step
    for _ in range(args.warmup):
        rc, lam, gam, info = gn_step(theta, lam, gam)
        if rc < 0:
            raise RuntimeError(f"gn_step failed in warm-up: {rc}")
    torch.cuda.synchronize()
    # the state the timed steps start from: the end-to-end run repeats exactly these steps
    theta_start, lam_start, gam_start = theta.clone(), lam, gam
    if world > 1:
        dist.barrier()
    L = gn.lib()
    launches0 = L.gn_kernel_launches()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    infos = []
    # a working set below the L2 size is flushed between timed steps (outside the events)
    flush = None
    if prob.n_rows * (prob.P + 1) * 8 < 512e6:
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    if flush is None:
        # one event between consecutive steps (each step synchronises anyway): the mean over the
        # timed region, plus the per-step median and interquartile range
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        evs[0].record(stream)
        for k in range(args.steps):
            rc, lam, gam, info = gn_step(theta, lam, gam)
            evs[k + 1].record(stream)
            if rc < 0:
                raise RuntimeError(f"gn_step failed: {rc}")
            infos.append(info)
        torch.cuda.synchronize()
        ms = evs[0].elapsed_time(evs[-1]) / args.steps
        per = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
        launches = L.gn_kernel_launches() - launches0
    else:
        per = []
        launches = 0
        for _ in range(args.steps):
            flush.fill_(1.0)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = L.gn_kernel_launches()
            ev0.record(stream)
            rc, lam, gam, info = gn_step(theta, lam, gam)
            ev1.record(stream)
            launches += L.gn_kernel_launches() - l0
            if rc < 0:
                raise RuntimeError(f"gn_step failed: {rc}")
            infos.append(info)
            torch.cuda.synchronize()
            per.append(ev0.elapsed_time(ev1))
        ms = statistics.mean(per)
    clocks = sampler.stop()
    if world > 1:
        ms = max_over_ranks(ms, "cuda")
        dist.barrier()
    value = world * 1000.0 / ms

    # per-phase device times (library CUDA events on the launch stream, averaged over the timed steps);
    # a captured graph is timed as a whole, so its phases come from eager steps of the same kernels
    # on a copy of the parameters, after the timed region
    phase_src = ("timed steps (CUDA events on the launch stream, recorded inside the graph as event nodes)"
                 if use_graph else "timed steps (library CUDA events on the launch stream)")
    phases = [statistics.mean(i["ms_phase"][k] for i in infos) for k in range(7)]
    if use_graph and phases[1] == 0.0:   # a streamed Jacobian carries no per-phase marks
        th2 = theta.clone()
        l2, g2, pinfos = lam, gam, []
        for _ in range(max(2, min(args.steps, 5))):
            rc2, l2, g2, i2 = prob.gn_step(th2, l2, g2)
            pinfos.append(i2)
        phases = [statistics.mean(i["ms_phase"][k] for i in pinfos) for k in range(7)]
        phase_src = f"{len(pinfos)} eager gn_step calls after the timed region (same kernels as the graph)"
    # the pipelined step (graph path) runs the Gram in column chunks beside the factorisation
    pipe_tiles = prob.gn_pipeline_tiles() if use_graph else 0
    kernels = kernel_report(prob, args, phases, pipe_tiles)
    # the roofline object describes the largest single kernel, the Gram launch (the Cholesky
    # phase is a chain of several kernels and is reported beside it under "kernels")
    roof = dict(kernels["gram"])

    # end to end through the C ABI with pinned host buffers: the same K steps again, from the
    # state the timed steps started from.  Every step copies theta in from pinned host memory,
    # steps, and copies theta back out with a blocking copy (the host holds the result before
    # the next step's input is formed from it); lambda, damping and the loss are host scalars
    # of the call.  The run must end on the timed run's final state bit for bit.
    e2e = None
    if not args.no_e2e:
        theta_dev_final, lam_dev_final, gam_dev_final = theta.clone(), lam, gam
        th_host = theta_start.detach().cpu().pin_memory()
        out_host = torch.empty_like(th_host).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lam2, gam2 = lam_start, gam_start
        for _ in range(args.steps):
            theta.copy_(th_host, non_blocking=True)
            rc, lam2, gam2, info2 = gn_step(theta, lam2, gam2)
            if rc < 0:
                raise RuntimeError(f"gn_step failed in the end-to-end run: {rc}")
            out_host.copy_(theta)            # blocking device-to-host copy of the step's result
            th_host.copy_(out_host)
        torch.cuda.synchronize()
        ms_e2e = (time.perf_counter() - t0) * 1e3 / args.steps
        same = bool(torch.equal(theta, theta_dev_final)) and lam2 == lam_dev_final and gam2 == gam_dev_final
        if not same:
            print("bench: the end-to-end run did not reproduce the device-timed run's final state",
                  file=sys.stderr)
        if world > 1:
            ms_e2e = max_over_ranks(ms_e2e, "cuda")
        nb = prob.P * 8
        e2e = {"value": world * 1000.0 / ms_e2e, "unit": UNIT, "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb, "ms_per_step": ms_e2e,
               "reproduces_timed_run": same,
               "note": "the timed run's K steps again from its starting state (host wall clock): theta in "
                       "from pinned host memory, gn_step through the C ABI, theta out to pinned host memory "
                       "with a blocking copy; lambda, damping and the loss are host scalars of the call"}

    # split precision vs FP64 at equal residual (CCF stable profile: the FP64 run's final validation
    # max |R| x 1.1 with its loss x 1.1 as the target), and
    # the batched sweep of 64 uneven fits as one graph launch per step
    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras["equal_residual"] = equal_residual_record("ccf_stable", args.extras_er_steps, "split_all", args.slices)
        b = batched_record(args, 5, 2)
        extras["batched"] = {k: b[k] for k in ("metric", "value", "unit", "ms_per_step", "steps", "warmup",
                                                "roofline", "gpu_launches")}
        extras["batched"]["config"] = b["config"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_step_estimate(workload=args.workload,
                                   budget_cols=12 if w.d == 1 else 3,
                                   gram_cols=512 if w.d == 1 else 256)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "ms_step_median": statistics.median(per),
                "ms_step_iqr": step_iqr(per), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": dict(workload_config(w, args.precision, args.slices),
                               **({"l2": "L2 flushed (256 MB write) between timed steps"} if flush is not None
                                  else {})),
                "roofline": roof, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": int(launches),
                "phase_ms": dict({"jacobian": phases[0], "gram": phases[1], "factor": phases[3],
                                  "solve": phases[4], "line_search": phases[5], "total": phases[6],
                                  "source": phase_src},
                                 **({"overlap": f"pipelined step (Gram chunks of {pipe_tiles} tiles): the gram "
                                                "and factor phases run at the same time"} if pipe_tiles else {})),
                "step_call": "gn_step_graph (captured CUDA graphs)" if use_graph else "gn_step",
                "final": {"loss": infos[-1]["loss_after"], "lambda": lam, "damping": gam,
                          "trials": [i["n_trials"] for i in infos]},
                **extras}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    prob.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
