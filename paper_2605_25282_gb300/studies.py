"""Studies on top of the library: the measurements and experiments of the
paper's Sec. 3-4 that are more than one bench step.

    python -m paper_2605_25282_gb300.studies ladder     [--precision fp64|mixed] [--steps 200]
    python -m paper_2605_25282_gb300.studies precision  [--nx 2560 --ny 1280 --M 64 --t 0.0035]
    python -m paper_2605_25282_gb300.studies cauchy     [--M 64 --times 0.0005,0.001,0.002,0.0035] [--batch 64]
    python -m paper_2605_25282_gb300.studies final      [--M 1000 --t 0.0035] [--save state.bin]
    python -m paper_2605_25282_gb300.studies resume     --load state.bin [--M 1000 --steps 200]
    python -m paper_2605_25282_gb300.studies adjoint    [--M 16 --steps 200 --limiter 2]
    python -m paper_2605_25282_gb300.studies stats      [--M 1000]

ladder     one realization per level of the single-realization refinement
           ladder (400x200 ... 5060x2530), fixed steps: cell-updates/s and
           achieved GB/s (algorithmic bytes / CUDA-event time) per level.
precision  seed-matched ensembles in the mixed path and in the FP64 path
           (whose update is the oracle's arithmetic) advanced to t with the
           landing rule (Sec. 2.3): per-field pathwise errors, per-statistic
           errors of rho and p, and W1 between the two ensembles along the jet
           axis; with --control, the same figures for two FP64 ensembles whose
           amplitudes differ by 1e-7 (the jet's own pathwise divergence).
cauchy     the paper's own ladder on [0, 2.5] x [-1, 1] (500x400 ... 4000x3200,
           Sec. 3.3) advanced together, with snapshots at the given times:
           every level's density restricted onto the coarsest grid, the error
           functionals of Sec. 3.4 (W_11, W_12, E_mean, E_std, E_strong) of the
           Cauchy and the reference comparisons, and their rates (Eq. (ratefit),
           least-squares slope in log-log).
final      the batched ensemble (M = 1000 of 400x200 + 800x400, mixed, one
           launch per step) to the paper's final time with the landing rule,
           then the statistics between the two levels; --save keeps the state.
resume     a saved state advanced a fixed number of steps (the step kernel on
           the developed, turbulent flow).
adjoint    the gradient configuration (512x256, checkpoints every 20 steps):
           time of the amplitude gradient against the forward steps alone.
stats      the statistics stage alone on the bench's levels (synthetic
           lognormal samples): time per call and achieved GB/s.

Every run prints one JSON object.  All inputs are synthetic and seeded
(Philox4x32-10 KL inlets, seed 0, realizations 0..M-1).
"""

from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import vlbm

BYTES_PER_UPDATE = {"fp64": 320, "mixed": 160}
LADDER_C2 = [(400, 200), (800, 400), (1600, 800), (3200, 1600), (5060, 2530)]
LADDER_PAPER = [(500, 400), (1000, 800), (2000, 1600), (4000, 3200)]


def _timed_steps(ens: vlbm.Ensemble, n: int) -> float:
    """Seconds of device time for n steps of every level, on the ensemble's stream."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(ens.stream):
        a.record(ens.stream)
        ens.step(n)
        b.record(ens.stream)
    b.synchronize()
    return a.elapsed_time(b) / 1e3


def ladder(precision: str = "fp64", steps: int = 200, warmup: int = 4, levels=LADDER_C2, M: int = 1,
           peak_gbs: float | None = None) -> dict:
    out = {"study": "refinement ladder, one realization per level", "precision": precision, "M": M,
           "steps": steps, "levels": []}
    for nx, ny in levels:
        ens = vlbm.Ensemble([(nx, ny)], precision=precision)
        ens.init(0, M)
        ens.step(warmup)
        sec = _timed_steps(ens, steps)
        cells = nx * ny * M * steps
        gbs = cells * BYTES_PER_UPDATE[precision] / sec / 1e9
        row = {"nx": nx, "ny": ny, "GLUPS": cells / sec / 1e9, "GBs": gbs, "ms_per_step": sec * 1e3 / steps,
               "state_MB": 2 * nx * ny * M * BYTES_PER_UPDATE[precision] / 2 / 1e6,
               "design": ens.step_design()[1], "rows_per_warp": ens.step_rows()}
        if peak_gbs:
            row["hbm_frac"] = gbs / peak_gbs
        # levels whose state fits in L2 (129 MB) are not HBM measurements
        row["l2_resident"] = row["state_MB"] * 2 < 129
        out["levels"].append(row)
        ens.sync()
        ens.close()
    return out


def _rel_l1(a: torch.Tensor, b: torch.Tensor, dims) -> torch.Tensor:
    return (a - b).abs().sum(dims) / b.abs().sum(dims)


def _pathwise(a: dict, b: dict) -> dict:
    """Realization-wise relative L1 differences of rho, u, v, p (median, max over m)."""
    out = {}
    for f in ("rho", "u", "v", "p"):
        if f in ("u", "v"):
            # velocities relative to the speed scale |v1| + |v2| of the reference field
            scale = (b["u"].abs() + b["v"].abs()).sum((1, 2))
            e = (a[f] - b[f]).abs().sum((1, 2)) / scale
        else:
            e = _rel_l1(a[f], b[f], (1, 2))
        out[f] = {"median": float(e.median()), "max": float(e.max())}
    return out


def _statistics(a: dict, b: dict, ny: int) -> dict:
    out = {}
    for f in ("rho", "p"):
        st = vlbm.stats_w1_mean_std(a[f], b[f])
        out[f] = {
            "mean": float((st["mean_a"] - st["mean_b"]).abs().sum() / st["mean_b"].abs().sum()),
            "std": float((st["std_a"] - st["std_b"]).abs().sum() / st["std_b"].abs().sum()),
            "w1_over_mean": float(st["w1"].sum() / st["mean_b"].abs().sum()),
        }
        if f == "rho":
            axis = st["w1"][ny // 2 - 1: ny // 2 + 1].mean(0)
            out["w1_axis_rho_mean"] = float(axis.mean())
    return out


def precision_study(nx: int = 2560, ny: int = 1280, M: int = 64, t: float = 0.0035, control: bool = False) -> dict:
    """Mixed against FP64, seed-matched.  With control, a third FP64 ensemble
    whose amplitudes differ by 1e-7 relative measures how far two precise
    runs drift apart by the same horizon (the pathwise divergence of the jet):
    the mixed path is as good as a precise path when its differences are of
    that size."""
    runs = {"mixed": ("mixed", vlbm.PerturbParams()), "fp64": ("fp64", vlbm.PerturbParams())}
    if control:
        amp = [0.1 * k ** -2.0 * (1.0 + 1e-7) for k in range(1, 11)]
        runs["fp64_perturbed"] = ("fp64", vlbm.PerturbParams(amp=amp))
    secs, steps, mo = {}, {}, {}
    for name, (prec, pert) in runs.items():
        e = vlbm.Ensemble([(nx, ny)], precision=prec)
        e.init(0, M, pert)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(e.stream):
            a.record(e.stream)
            e.advance_to(t)
            b.record(e.stream)
        b.synchronize()
        secs[name] = a.elapsed_time(b) / 1e3
        steps[name] = e.time(0)[1]
        mo[name] = e.moments(0)
        e.close()
    out = {"study": "precision: mixed vs FP64, seed-matched", "nx": nx, "ny": ny, "M": M, "t": t,
           "steps": {p: [int(s.min()), int(s.max())] for p, s in steps.items()},
           "seconds": secs,
           "cell_updates_per_s": {p: float(nx * ny * steps[p].sum() / secs[p]) for p in secs},
           "mixed_vs_fp64": {"pathwise_rel_l1": _pathwise(mo["mixed"], mo["fp64"]),
                             "statistics_rel_l1": _statistics(mo["mixed"], mo["fp64"], ny)}}
    if control:
        out["fp64_perturbed_vs_fp64"] = {"amplitude_change": 1e-7,
                                         "pathwise_rel_l1": _pathwise(mo["fp64_perturbed"], mo["fp64"]),
                                         "statistics_rel_l1": _statistics(mo["fp64_perturbed"], mo["fp64"], ny)}
    return out


def rate(h, err) -> float | None:
    """Least-squares slope of log err against log h (None if any err <= 0)."""
    h, err = np.asarray(h, float), np.asarray(err, float)
    if len(h) < 2 or np.any(err <= 0):
        return None
    return float(np.polyfit(np.log(h), np.log(err), 1)[0])


def _functionals(a: torch.Tensor, b: torch.Tensor, npd: int = 10, w12: bool = True) -> dict:
    f = vlbm.stats_error_functionals(a, b)
    e_mean, e_std, w11, e_strong = (float(x) for x in f.cpu())
    out = {"W_11": w11, "E_mean": e_mean, "E_std": e_std, "E_strong": e_strong}
    if w12:
        out["W_12"] = float(vlbm.stats_w1_two_point(a, b, npd)[0])
    return out


def axial_profile(axis: torch.Tensor, x_max: float = 2.5, rho_amb: float = 0.5) -> dict:
    """Ensemble statistics of the density on the jet axis of one level, from
    its two rows next to y = 0 ([M, 2, nx]): the bow-shock position (the
    largest x where the axial mean exceeds the ambient density by 10 %), the
    median axial std upstream of x = 1.4, and the peak axial std with the mean
    there (the quantities Sec. 4 reads off the axis); population std."""
    M, _, nx = axis.shape
    a = axis.double()
    mean = a.mean(0).mean(0).cpu().numpy()
    std = a.std(0, unbiased=False).mean(0).cpu().numpy()
    x = np.arange(nx) * (x_max / nx)
    above = np.nonzero(mean > 1.1 * rho_amb)[0]
    k = int(np.argmax(std))
    return {"bow_shock_x": float(x[above[-1]]) if len(above) else 0.0,
            "axial_std_upstream_median": float(np.median(std[(x > 0.05) & (x < 1.4)])),
            "axial_std_peak": float(std[k]), "axial_std_peak_x": float(x[k]), "axial_mean_at_peak": float(mean[k])}


def cauchy(M: int = 64, times=(0.0005, 0.001, 0.002, 0.0035), levels=LADDER_PAPER, precision: str = "mixed",
           batch: int | None = None, w12: bool = True) -> dict:
    """The paper's protocol (Sec. 3.3-3.4): every level's density restricted
    onto the coarsest grid, the Cauchy comparison of successive levels and the
    reference comparison against the finest, rates by Eq. (ratefit).  The M
    realizations run in batches of `batch` (realizations b .. b + batch - 1
    of the same seeded sequence, all four levels in one launch per step); the
    restricted densities and the axis rows of every batch are kept in host
    memory and the functionals are taken over all M at the end.  W_12 (an
    exact M-point assignment per point pair) is skipped with w12 False."""
    batch = min(batch or M, M)
    nx0, ny0 = levels[0]
    T, NL = len(times), len(levels)
    keep = {(ti, l): [] for ti in range(T) for l in range(NL)}
    axis_rows = {(ti, l): [] for ti in range(T) for l in range(NL)}
    secs = [0.0] * T
    steps = [[None] * NL for _ in range(T)]
    for b0 in range(0, M, batch):
        mb = min(batch, M - b0)
        ens = vlbm.Ensemble(levels, precision=precision)
        ens.init(0, mb, m_begin=b0)
        for ti, t in enumerate(times):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(ens.stream):
                a.record(ens.stream)
                ens.advance_to(t)
                b.record(ens.stream)
            b.synchronize()
            secs[ti] += a.elapsed_time(b) / 1e3
            for l, (nx, ny) in enumerate(levels):
                s_l = ens.time(l)[1]
                lo, hi = int(s_l.min()), int(s_l.max())
                prev = steps[ti][l]
                steps[ti][l] = [lo, hi] if prev is None else [min(prev[0], lo), max(prev[1], hi)]
                # the binding orders the caller's current stream after the
                # ensemble's work; restriction then runs on that stream
                d = ens.density(l, f32=False)
                axis_rows[(ti, l)].append(d[:, ny // 2 - 1: ny // 2 + 1].float().cpu())
                c = vlbm.stats_restrict(d, nx // nx0) if nx != nx0 else d
                keep[(ti, l)].append(c.cpu())
                del d, c
        ens.close()
    out = {"study": "Cauchy and reference convergence on the paper's ladder", "domain": "[0, 2.5] x [-1, 1]",
           "M": M, "batch": batch, "precision": precision, "levels": [list(lv) for lv in levels],
           "common_grid": [nx0, ny0], "snapshots": []}
    keys = ("W_11", "W_12", "E_mean", "E_std", "E_strong") if w12 else ("W_11", "E_mean", "E_std", "E_strong")
    L = NL - 1
    dx = [2.5 / nx for nx, _ in levels]
    for ti, t in enumerate(times):
        common = [torch.cat(keep[(ti, l)]).cuda() for l in range(NL)]
        axis = [axial_profile(torch.cat(axis_rows[(ti, l)])) for l in range(NL)]
        snap = {"t": t, "seconds": secs[ti], "steps": steps[ti], "axis": axis, "cauchy": [], "reference": []}
        for l in range(1, L + 1):
            snap["cauchy"].append({"pair": [levels[l - 1][0], levels[l][0]],
                                   **_functionals(common[l - 1], common[l], w12=w12)})
        for l in range(L):
            snap["reference"].append({"pair": [levels[l][0], levels[L][0]],
                                      **_functionals(common[l], common[L], w12=w12)})
        snap["rates"] = {
            "cauchy": {k: rate(dx[:L], [p[k] for p in snap["cauchy"]]) for k in keys},
            "reference": {k: rate(dx[:L], [p[k] for p in snap["reference"]]) for k in keys},
        }
        out["snapshots"].append(snap)
        del common
    return out


def batched_final_time(M: int = 1000, t: float = 0.0035, levels=((400, 200), (800, 400)),
                       save: str | None = None, precision: str = "mixed") -> dict:
    """The batched ensemble run to the paper's final time: M realizations of
    both levels in one launch per step (mixed, landing on t), then the
    per-cell mean, std and one-point W1 between the levels (the fine level
    restricted onto the coarse grid) and the error functionals."""
    levels = [tuple(lv) for lv in levels]
    ens = vlbm.Ensemble(levels, precision=precision)
    ens.init(0, M)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(ens.stream):
        a.record(ens.stream)
        ens.advance_to(t)
        b.record(ens.stream)
    b.synchronize()
    sec = a.elapsed_time(b) / 1e3
    steps = [ens.time(l)[1] for l in range(len(levels))]
    times = [ens.time(l)[0] for l in range(len(levels))]
    cells = sum(nx * ny * int(s.sum()) for (nx, ny), s in zip(levels, steps))
    d0, d1 = ens.density(0), ens.density(1)
    a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a2.record()
    st = vlbm.stats_w1_mean_std(d0, d1)
    b2.record()
    b2.synchronize()
    f = _functionals(d0, d1)
    out = {"study": "batched ensemble to the final time", "M": M, "t": t, "levels": [list(lv) for lv in levels],
           "precision": precision, "design": ens.step_design()[1], "seconds": sec, "cell_updates": cells,
           "GLUPS": cells / sec / 1e9, "steps": [[int(s.min()), int(s.max())] for s in steps],
           "t_reached": [[float(x.min()), float(x.max())] for x in times],
           "stats_ms": a2.elapsed_time(b2),
           "mean_rho_range": [float(st["mean_a"].min()), float(st["mean_a"].max())],
           "max_std_rho": float(st["std_a"].max()), "w1_cell_mean": float(st["w1"].mean()),
           "functionals_coarse_vs_fine": f}
    if save:
        with open(save, "wb") as fh:
            fh.write(ens.save())
        out["saved"] = save
    ens.close()
    return out


def resume_steps(load: str, M: int, steps: int, levels=((400, 200), (800, 400)), precision: str = "mixed") -> dict:
    """Restores a state written by `final --save` (same levels, M and precision)
    and advances it `steps` fixed steps: the step kernel on a developed flow."""
    levels = [tuple(lv) for lv in levels]
    ens = vlbm.Ensemble(levels, precision=precision)
    ens.init(0, M)
    with open(load, "rb") as fh:
        ens.load(fh.read())
    t0 = [ens.time(l) for l in range(len(levels))]
    sec = _timed_steps(ens, steps)
    cells = sum(nx * ny for nx, ny in levels) * M * steps
    out = {"study": "steps on a restored state", "M": M, "levels": [list(lv) for lv in levels], "steps": steps,
           "t_start": [float(t[0].min()) for t in t0], "seconds": sec, "GLUPS": cells / sec / 1e9,
           "GBs": cells * BYTES_PER_UPDATE[precision] / sec / 1e9, "precision": precision,
           "design": ens.step_design()[1]}
    ens.close()
    return out


def adjoint_timing(nx: int = 512, ny: int = 256, M: int = 16, steps: int = 200, every: int = 20,
                   limiter: int = 2) -> dict:
    """The adjoint configuration: the gradient of the axial ensemble-mean density
    after `steps` FP64 steps with respect to the KL amplitudes (checkpoints every
    `every` steps), timed against the forward steps alone."""
    ens = vlbm.Ensemble([(nx, ny)], precision="fp64", relax=vlbm.RelaxParams(limiter=limiter))
    ens.init(0, M)
    w = vlbm.axial_weights(ny, nx)
    ens.grad_amplitudes(2, w, every)  # warm-up (tuning, allocations)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(ens.stream):
        a.record(ens.stream)
        J, grad = ens.grad_amplitudes(steps, w, every)
        b.record(ens.stream)
    b.synchronize()
    sec = a.elapsed_time(b) / 1e3
    ens.init(0, M)
    fwd = _timed_steps(ens, steps)
    cells = nx * ny * M * steps
    out = {"study": "adjoint: gradient of the axial ensemble-mean density", "nx": nx, "ny": ny, "M": M,
           "steps": steps, "checkpoint_every": every, "limiter": limiter, "J": J, "grad": [float(g) for g in grad],
           "seconds_gradient": sec, "seconds_forward": fwd, "gradient_over_forward": sec / fwd,
           "forward_GLUPS": cells / fwd / 1e9, "design": ens.step_design()[1]}
    ens.close()
    return out


def stats_timing(M: int = 1000, levels=((400, 200), (800, 400)), reps: int = 10) -> dict:
    """The statistics stage alone on the bench's levels: restriction of the fine
    level, per-cell mean, std and sorted one-point W1 over M samples (FP32
    inputs, lognormal densities around the jet's values), CUDA-event time."""
    (nxa, nya), (nxb, nyb) = levels
    g = torch.Generator(device="cuda").manual_seed(0)
    a = torch.exp(0.3 * torch.randn((M, nya, nxa), device="cuda", generator=g)).float()
    b = torch.exp(0.3 * torch.randn((M, nyb, nxb), device="cuda", generator=g)).float()
    for _ in range(3):
        vlbm.stats_w1_mean_std(a, b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        vlbm.stats_w1_mean_std(a, b)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    r = nxb // nxa
    nbytes = nxa * nya * (M * 4 * (1 + r * r) + 5 * 8)
    return {"study": "statistics stage alone", "M": M, "levels": [list(lv) for lv in levels], "ms_per_call": ms,
            "bytes_per_call": nbytes, "GBs": nbytes / (ms / 1e3) / 1e9}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("study", choices=["ladder", "precision", "cauchy", "final", "resume", "adjoint", "stats"])
    ap.add_argument("--precision", choices=["fp64", "mixed"], default=None)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--M", type=int, default=None)
    ap.add_argument("--nx", type=int, default=2560)
    ap.add_argument("--ny", type=int, default=1280)
    ap.add_argument("--t", type=float, default=0.0035, help="final time (precision study)")
    ap.add_argument("--times", type=str, default="0.0005,0.001,0.002,0.0035", help="snapshot times (cauchy)")
    ap.add_argument("--peak-gbs", type=float, default=None)
    ap.add_argument("--levels", type=str, default=None,
                    help="ladder: levels as NXxNY,... (default: the refinement ladder 400x200 ... 5060x2530)")
    ap.add_argument("--warmup", type=int, default=4, help="ladder: untimed steps before the timed ones")
    ap.add_argument("--limiter", type=int, default=2, help="adjoint: 0 = theta 0 (Lax-Friedrichs), 2 = R-theta")
    ap.add_argument("--batch", type=int, default=None, help="cauchy: realizations per batch (default: all at once)")
    ap.add_argument("--no-w12", action="store_true", help="cauchy: skip the two-point distance W_12")
    ap.add_argument("--control", action="store_true", help="precision: add a perturbed FP64 control run")
    ap.add_argument("--save", type=str, default=None, help="final: write the final state to this file")
    ap.add_argument("--load", type=str, default=None, help="resume: the state file written by final --save")
    args = ap.parse_args(argv)
    if args.study == "ladder":
        levels = LADDER_C2 if not args.levels else [tuple(int(v) for v in lv.split("x")) for lv in args.levels.split(",")]
        res = ladder(args.precision or "fp64", args.steps, warmup=args.warmup, levels=levels, M=args.M or 1,
                     peak_gbs=args.peak_gbs)
    elif args.study == "precision":
        res = precision_study(args.nx, args.ny, args.M or 64, args.t, args.control)
    elif args.study == "cauchy":
        res = cauchy(args.M or 64, [float(x) for x in args.times.split(",")], precision=args.precision or "mixed",
                     batch=args.batch, w12=not args.no_w12)
    elif args.study == "final":
        res = batched_final_time(args.M or 1000, args.t, save=args.save, precision=args.precision or "mixed")
    elif args.study == "adjoint":
        res = adjoint_timing(M=args.M or 16, steps=args.steps, limiter=args.limiter)
    elif args.study == "stats":
        res = stats_timing(M=args.M or 1000)
    else:
        res = resume_steps(args.load, args.M or 1000, args.steps, precision=args.precision or "mixed")
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
