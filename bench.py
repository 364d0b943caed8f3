"""Benchmark of the probabilistic VLBM hot path on GB300.

One bench step is one pass of the whole path over one batch: seeded ensemble
initialisation (Philox + KL inlet, initial condition), S VLBM steps of every
realization on both grid levels (kinetic speed, primitive recovery,
Maxwellians, first-order state, faces and limiter, fused update + stream,
boundaries), density extraction of both levels and the per-cell statistics
between the levels (restriction, mean, std, one-point W1 from a per-cell sort).

Workload (default): the batched ensemble of M = 1000 jet realizations per GPU
on the 400 x 200 and 800 x 400 levels in one launch per step, mixed precision.
Metric: ensemble cell-updates per second (GLUPS) = sum over levels and
realizations of nx ny x S / wall seconds of the bench step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

LEVELS = [(400, 200), (800, 400)]
M_PER_GPU = 1000
SEED = 0
METRIC = "ensemble cell-updates/s (GLUPS) & % HBM roofline, mixed vs FP64, at stated stat error"
BYTES_PER_UPDATE = {"mixed": 160, "fp64": 320}
# DRAM traffic of one step-kernel launch from an ncu capture, with the sha256
# of the kernel source and the launch design it was taken on (reported as null
# once either differs).  Mixed: 607.0 MB read + written for the 4.0 M
# cell-updates of the M = 10 capture (333.3 MB read + 273.6 MB written),
# scaled to 400 M cell-updates.
NCU_TRAFFIC = {
    "mixed": {"sha": "0d90d89fd786c14a", "design": "march30pf4w", "bytes_per_launch": 60.70e9,
              "capture": "M=10, 400x200 + 800x400, scaled by cell-updates"},
}
# The FP64 step kernel is bound by the FP64 pipe, not by HBM.  ncu counters of
# the warp-march design on M = 2 realizations of 400x200 + 800x400 (800,000
# cell-updates per launch), with the sha256 of the kernel source and of its
# math header: FP64-pipe warp instructions x 32 per cell-update (every FP64
# add, multiply, fused multiply-add, compare, min/max and conversion; the FP64
# pipe runs all 32 lanes of a warp instruction) and the FLOPs of the adds,
# multiplies and fused multiply-adds, on the first steps of a run (151.0 M
# DADD + 149.5 M DMUL + 108.9 M DFMA) and on the developed flow at t = 0.002
# (157.4 M DADD + 146.5 M DMUL + 73.2 M DFMA).  A full run is mostly developed
# flow, so the roofline uses the developed count.  GB300 issues 2 FP64 thread
# operations per SM and clock (152 x 2 x 2 x 2.07 GHz = 1.26 TFLOP/s, GB300's
# nominal FP64 rate).
FP64_ALU = {"sha": "24e738279663953b+ce7574c07d3d6886",
            "pipe_inst_per_update": 15484412 * 32 / 800000,
            "pipe_inst_per_update_first_steps": 15645124 * 32 / 800000,
            "flop_per_update": (157408760 + 146507958 + 2 * 73170058) / 800000, "ops_per_sm_clock": 2,
            "sms": 152}


def peaks():
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_sha(precision: str) -> str:
    names = ["vlbm_step_mixed.cu"] if precision == "mixed" else ["vlbm_step_f64.cu", "vlbm_f64_math.cuh"]
    out = []
    for name in names:
        with open(os.path.join(HERE, "paper_2605_25282_gb300", "csrc", name), "rb") as f:
            out.append(hashlib.sha256(f.read()).hexdigest()[:16])
    return "+".join(out)


def sm_max_mhz() -> float:
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return 2070.0


def fp64_alu(glups: float):
    """ALU roofline of the FP64 step kernel at `glups` G cell-updates/s (None
    once the kernel source differs from the one the counters were taken on)."""
    if kernel_sha("fp64") != FP64_ALU["sha"]:
        return None
    mhz = sm_max_mhz()
    peak = FP64_ALU["sms"] * FP64_ALU["ops_per_sm_clock"] * mhz * 1e6 / 1e9
    achieved = glups * FP64_ALU["pipe_inst_per_update"]
    return {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": peak, "unit": "G FP64 inst/s",
            "frac": achieved / peak, "inst_per_cell_update": FP64_ALU["pipe_inst_per_update"],
            "inst_per_cell_update_first_steps": FP64_ALU["pipe_inst_per_update_first_steps"],
            "flop_per_cell_update": FP64_ALU["flop_per_update"],
            "peak_source": f"{FP64_ALU['sms']} SMs x {FP64_ALU['ops_per_sm_clock']} FP64 ops per clock x "
                           f"{mhz:.0f} MHz (sm_max_mhz)"}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for s in self.samples for n, v in zip(names, s[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_setup(gpus: int):
    """Rank, world size and local GPU from the launcher's environment (one
    process per GPU under torchrun; without it a single rank).  The world size
    is the launcher's: --gpus N without torchrun runs and reports one GPU."""
    rank = int(os.environ.get("RANK", "0"))
    world = max(int(os.environ.get("WORLD_SIZE", "1")), 1)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != gpus and rank == 0:
        print(f"bench: --gpus {gpus} but {world} process(es) launched; reporting {world}", file=sys.stderr)
    return rank, world, local


def _oracle_task(args):
    """One realization of every level, `steps` oracle steps, and its statistics
    (runs in a worker process)."""
    levels, steps, m = args
    from oracle import oracle as O

    dens = []
    cells = 0
    for (nx, ny) in levels:
        r = O.run_jet(O.Grid(nx, ny), O.Params(), O.Jet(), SEED, m, 1, steps, want_pops=False)
        dens.append(r["u"][:, 0])
        cells += nx * ny * steps
    O.stats_w1_mean_std(dens[0], dens[1])
    return cells


class OraclePool:
    """The oracle (plain FP64 C, one thread per process) on the host's cores:
    one realization per worker process, all workers at once."""

    def __init__(self, workers: int | None = None):
        import concurrent.futures
        import multiprocessing

        self.workers = workers or os.cpu_count() or 1
        self.ex = concurrent.futures.ProcessPoolExecutor(self.workers,
                                                         mp_context=multiprocessing.get_context("spawn"))
        # start every worker (imports, library load) outside any timing
        list(self.ex.map(_oracle_task, [([(8, 4), (16, 8)], 1, w) for w in range(self.workers)]))

    def rate(self, levels, steps: int, m0: int = 0):
        t0 = time.perf_counter()
        cells = sum(self.ex.map(_oracle_task, [(levels, steps, m0 + w) for w in range(self.workers)]))
        dt = time.perf_counter() - t0
        return cells / dt / 1e9, dt, cells

    def close(self):
        self.ex.shutdown()


def horizon_of(args) -> str:
    if args.t_final > 0:
        return (f"to the next output time t_k = k x {args.dt_snap} (landing rule; a fresh ensemble after "
                f"t = {args.t_final})")
    return f"{args.solver_steps} VLBM steps"


def workload_config(levels, M, horizon, prec):
    nxa = " + ".join(f"{nx}x{ny}" for nx, ny in levels)
    state_gb = sum(nx * ny for nx, ny in levels) * M * BYTES_PER_UPDATE[prec] / 1e9
    return {"workload": f"Mach 2000 jet ensemble, M={M} per GPU, levels {nxa} in one launch, {prec}, R-theta "
                        f"limiter, per bench step: every realization {horizon} + density + W1/mean/std "
                        f"statistics between the levels",
            "levels": levels, "M_per_gpu": M, "horizon": horizon, "precision": prec,
            "l2": f"inputs {'larger' if state_gb > 0.129 else 'SMALLER'} than L2 (lattice state "
                  f"{state_gb:.3g} GB)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    levels = LEVELS
    per = 6  # oracle steps of each realization per bench step
    pool = OraclePool()
    for w in range(args.warmup):
        pool.rate(levels, per, m0=w * pool.workers)
    times = []
    cells = 0
    for k in range(args.steps):
        _, dt, c = pool.rate(levels, per, m0=(args.warmup + k) * pool.workers)
        times.append(dt)
        cells += c
    pool.close()
    total = sum(times)
    value = cells / total / 1e9
    sample = (f"{pool.workers} realizations (one per host core, one process each) x "
              f"({' + '.join(f'{nx}x{ny}' for nx, ny in levels)}) x {per} VLBM steps per bench step, plus the "
              "statistics of each; FP64 oracle")
    line = {
        "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Philox jet ensemble)",
        "impl": "reference",
        "config": workload_config(levels, args.m, horizon_of(args), args.precision),
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": pool.workers, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _stat_errors(vlbm, a, b, stream):
    """L1-normalised errors of the per-cell mean and std of ensemble a against
    ensemble b, and their one-point W1 over sum |mean_b| (Sec. 3.2)."""
    st = vlbm.stats_w1_mean_std(a, b, stream=stream)
    ma, sa, mb, sb, w1 = (st[k].double() for k in ("mean_a", "std_a", "mean_b", "std_b", "w1"))
    return {"mean": float((ma - mb).abs().sum() / mb.abs().sum()),
            "std": float((sa - sb).abs().sum() / sb.abs().sum()),
            "w1": float(w1.sum() / mb.abs().sum())}


def precision_legs(vlbm, levels, args, stream, m_begin):
    """Seed-matched ensembles of M = stat_m realizations: the mixed path, the
    FP64 path on 2M realizations (the second half an independent ensemble of
    the same size: the Monte-Carlo error at matched M) and an FP64 control
    whose KL amplitudes differ by 1e-7 relative (the jet's own pathwise
    divergence from a perturbation of FP32 size).  Statistic errors after 64
    steps and at the final time; the FP64 and mixed rates over the same run."""
    import torch

    M = args.stat_m
    horizon = args.t_final if args.t_final > 0 else None
    amp = [0.1 * k ** -2.0 * (1.0 + 1e-7) for k in range(1, 11)]
    runs = {"mixed": ("mixed", M, vlbm.PerturbParams()), "fp64": ("fp64", 2 * M, vlbm.PerturbParams()),
            "control": ("fp64", M, vlbm.PerturbParams(amp=amp))}
    dens, rates = {}, {}
    for name, (p, m, pert) in runs.items():
        for phase, n in (("short", 64), ("final", None)):
            e = vlbm.Ensemble(levels, precision=p, stream=stream)
            e.init(SEED, m, pert, m_begin=m_begin)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if n is not None:
                e.step(n)
            elif horizon is not None:
                e.advance_to(horizon)
            else:
                e.step(args.solver_steps)
            b.record(stream)
            b.synchronize()
            if phase == "final":
                cells = sum(nx * ny * int(e.time(l)[1].sum()) for l, (nx, ny) in enumerate(levels))
                rates[name] = {"value": cells / (a.elapsed_time(b) / 1e3) / 1e9, "M": m,
                               "cell_updates": cells, "seconds": a.elapsed_time(b) / 1e3}
            dens[(name, phase)] = [e.density(l, f32=False) for l in range(len(levels))]
            e.close()
    out = {"M": M, "norm": "sum over cells |s - s_ref| / sum |s_ref| (W1 between the ensembles: / sum |mean_ref|); "
                           "the fine level restricted onto the coarse grid is not used: each level on its own",
           "reference": "FP64 path (the oracle's arithmetic, equal to the oracle to 1e-12 per cell over 10 steps), "
                        "same seed and realizations"}
    for phase, label in (("short", "64 steps"), ("final", f"t = {horizon}" if horizon else "final")):
        row = {"horizon": label}
        for l, lname in enumerate(("coarse", "fine")):
            ref = dens[("fp64", phase)][l][:M]
            row[lname] = {
                "mixed_vs_fp64": _stat_errors(vlbm, dens[("mixed", phase)][l], ref, stream),
                "fp64_control_vs_fp64": _stat_errors(vlbm, dens[("control", phase)][l], ref, stream),
                "independent_fp64_vs_fp64": _stat_errors(vlbm, dens[("fp64", phase)][l][M:], ref, stream)}
        out[phase] = row
    fp64 = {"value": rates["fp64"]["value"], "unit": "GLUPS", "M": rates["fp64"]["M"],
            "horizon": "t = 0 to the final time (landing rule), the bench run's horizon",
            "seconds": rates["fp64"]["seconds"], "mixed_same_run": rates["mixed"]}
    return fp64, out


def run_ours(args):
    import torch

    from paper_2605_25282_gb300 import sharded, vlbm

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = tdist
    dev = torch.device("cuda", local)
    # every launch of the bench runs on one non-default stream: the library's
    # kernels, the statistics, the copies and the CUDA events
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    levels = LEVELS
    M = args.m
    S = args.solver_steps
    prec = args.precision
    ens = vlbm.Ensemble(levels, precision=prec, stream=stream)
    m_begin = rank * M
    horizon = horizon_of(args)
    (nxa, nya), (nxb, nyb) = levels
    dens_a = torch.empty((M, nya, nxa), dtype=torch.float32, device=dev)
    dens_b = torch.empty((M, nyb, nxb), dtype=torch.float32, device=dev)
    host_out = [torch.empty((nya, nxa), dtype=torch.float64, pin_memory=True) for _ in range(5)]
    # end-to-end inputs: the KL coefficients of every realization (Sec. 2.3,
    # Eq. (karhunenExp)), uniform on (-1, 1), in pinned host memory
    K = vlbm.PerturbParams().K
    rng = np.random.default_rng(SEED + rank)
    host_xi = torch.from_numpy(rng.uniform(-1.0, 1.0, (M, 2 * K))).pin_memory()

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    step_ms = []
    stats_ms = []

    # A bench step advances every realization to the next of the paper's
    # output times (every dt_snap up to t_final, landing rule) and takes the
    # statistics between the levels there; after t_final the next step starts
    # from a fresh ensemble.  A cycle of n_snap steps is one full run.
    n_snap = max(1, int(round(args.t_final / args.dt_snap))) if args.t_final > 0 else 1
    phase = {"k": n_snap}  # snapshot index of the state held (n_snap: start a new run)

    def steps_now():
        return [ens.time(l)[1].copy() for l in range(len(levels))]

    def bench_step(e2e: bool, timed: bool):
        if phase["k"] >= n_snap:
            if e2e:
                ens.init_samples(host_xi)
            else:
                ens.init(SEED, M, m_begin=m_begin)
            phase["k"] = 0
        before = steps_now() if phase["k"] > 0 else [np.zeros(M, dtype=np.int64) for _ in levels]
        if timed:
            ev[0].record(stream)
        if args.t_final > 0:
            ens.advance_to(args.t_final * (phase["k"] + 1) / n_snap)
        else:
            ens.step(S)
        if timed:
            ev[1].record(stream)
        phase["k"] += 1
        ens.density(0, out=dens_a)
        ens.density(1, out=dens_b)
        if timed:
            ev[2].record(stream)
        if dist is None:
            st = vlbm.stats_w1_mean_std(dens_a, dens_b, stream=stream)
        else:
            # statistics over the realizations of every rank: one row-block all-to-all
            st = sharded.gpu_statistics(dens_a, dens_b)
        if timed:
            ev[3].record(stream)
        if e2e:
            for h, k in zip(host_out, ("mean_a", "std_a", "mean_b", "std_b", "w1")):
                h.copy_(st[k], non_blocking=True)
            stream.synchronize()  # the caller reads the statistics of this step
        after = steps_now()
        return sum(nx * ny * int((a - b).sum()) for (nx, ny), a, b in zip(levels, after, before))

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def timed_loop(e2e: bool, warmup: int):
        for _ in range(warmup):
            bench_step(e2e, False)
        barrier()
        launches0 = vlbm.kernel_launches()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        h0 = time.perf_counter()
        t0.record(stream)
        cells = 0
        for _ in range(args.steps):
            cells += bench_step(e2e, not e2e)
            if not e2e:
                step_ms.append(ev[0].elapsed_time(ev[1]))
                stats_ms.append(ev[2].elapsed_time(ev[3]))
        t1.record(stream)
        barrier()
        # device time for the kernel-only figure; host wall time end to end
        ms = t0.elapsed_time(t1) if not e2e else (time.perf_counter() - h0) * 1e3
        launches = vlbm.kernel_launches() - launches0
        if dist is not None:
            tt = torch.tensor([ms, float(cells)], dtype=torch.float64, device=dev)
            mx = tt.clone()
            dist.all_reduce(mx, op=dist.ReduceOp.MAX)
            dist.all_reduce(tt, op=dist.ReduceOp.SUM)
            ms, cells_all = float(mx[0].item()), int(tt[1].item())
        else:
            cells_all = cells
        return ms, launches, cells, cells_all

    clocks = ClockSampler(local)
    clocks.start()
    ms, launches, cells_timed, cells_all = timed_loop(False, args.warmup)
    clk = clocks.stop()
    # the system is warm: one untimed end-to-end step, then the timed ones
    phase["k"] = n_snap
    ms_e2e, _, _, cells_all_e2e = timed_loop(True, 1)
    design = ens.step_design()

    # The FP64 path (the oracle's arithmetic) and the statistic errors, on the
    # bench's own horizon: seed-matched ensembles of the same levels run from
    # t = 0 to the final time with the landing rule, like one bench run.
    fp64, stat_err = None, None
    if args.stat_m > 0 and prec == "mixed":
        fp64, stat_err = precision_legs(vlbm, levels, args, stream, m_begin)
    value = cells_all / (ms / 1e3) / 1e9
    e2e_value = cells_all_e2e / (ms_e2e / 1e3) / 1e9
    hbm, src = peaks()
    if fp64 is not None:
        fp64["hbm_frac"] = fp64["value"] * 1e9 * BYTES_PER_UPDATE["fp64"] / (hbm * 1e9)
        fp64["alu"] = fp64_alu(fp64["value"])
    # the step kernels of the timed bench steps: algorithmic bytes of their
    # cell-updates over the CUDA-event time of the advances (ticks, landing
    # and the polling of active realizations included)
    adv_s = float(np.sum(step_ms)) / 1e3
    achieved = BYTES_PER_UPDATE[prec] * cells_timed / adv_s / 1e9
    sha = kernel_sha(prec)
    tr = NCU_TRAFFIC.get(prec)
    traffic = tr["bytes_per_launch"] if tr and tr["sha"] == sha and tr["design"] == design[1] else None
    if prec == "mixed":
        kname = {"tile": "step_mixed_tile_kernel", "pers": "step_mixed_persistent_kernel",
                 "marc": "step_mixed_march_kernel"}.get(design[1][:4], "step_mixed_kernel")
    else:
        kname = "step_f64_march_kernel" if design[1].startswith("march") else "step_f64_kernel"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic,
                "kernel": kname, "design": design[1], "peak_source": f"{src} hbm_gbs",
                "bytes_per_cell_update": BYTES_PER_UPDATE[prec],
                "advance_ms": adv_s * 1e3,
                "note": f"achieved = {BYTES_PER_UPDATE[prec]} B x cell-updates of the timed bench steps / "
                        "CUDA-event time of their advances (every step launch, tick and landing check; "
                        "realizations that landed leave the launches); traffic: ncu DRAM bytes of one launch "
                        "with every realization active"}
    # the statistics call of each timed step (restriction of the fine level,
    # per-cell mean, std and sorted W1): read (1 + r^2) M FP32 samples and
    # write 5 FP64 fields per coarse cell
    r = nxb // nxa
    # (one GPU; sharded, the call also restricts, exchanges and gathers)
    stats_bytes = nxa * nya * (M * 4 * (1 + r * r) + 5 * 8) if dist is None else None
    stats_s = float(np.mean(stats_ms)) / 1e3
    stats_gbs = stats_bytes / stats_s / 1e9 if stats_bytes else None
    stats = {"kernel": "stats_kernel", "ms_per_call": stats_s * 1e3, "bytes_per_call": stats_bytes,
             "achieved_gbs": stats_gbs, "hbm_frac": stats_gbs / hbm if stats_gbs else None,
             "share_of_step": stats_s * 1e3 / (ms / args.steps),
             "bound": "FP64 pipe (ncu: 80 % busy with the samples' FP64 conversions, restriction sums and "
                      "moments; the per-cell sort runs on integer order keys)",
             "sharded": dist is not None}
    if prec == "fp64":
        # bound by the FP64 pipe: the roofline is the ALU one, the HBM figures stay beside it
        alu = fp64_alu(cells_timed / adv_s / 1e9)
        if alu is not None:
            roofline = {**alu, "kernel": kname, "design": design[1], "advance_ms": adv_s * 1e3,
                        "hbm": {"achieved_gbs": achieved, "frac": achieved / hbm, "traffic": traffic}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        pool = OraclePool()
        r, dt, c = pool.rate(levels, args.cpu_steps)
        cpu = {"value": r, "unit": "GLUPS", "cores": pool.workers, "kind": "oracle",
               "sample": f"{pool.workers} realizations (one process per host core) x (400x200 + 800x400) x "
                         f"{args.cpu_steps} VLBM steps + statistics, {dt:.1f} s wall"}
        pool.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == "mixed" else "f64",
            "data": "synthetic (seeded Philox4x32-10 Karhunen-Loeve jet inlets)",
            "config": {**workload_config(levels, M, horizon, prec), "snapshots_per_run": n_snap,
                       "cell_updates_timed": cells_timed},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "GLUPS", "h2d_bytes_per_step": M * 2 * K * 8 / n_snap,
                    "d2h_bytes_per_step": 5 * nxa * nya * 8,
                    "note": f"host wall clock through the public API: the first step of every run (one in "
                            f"{n_snap}) copies the KL coefficients of all realizations ({M * 2 * K * 8} B) from "
                            "pinned host memory (vlbm_init_ensemble_samples); every step advances and reads "
                            "the statistics back to pinned host memory; h2d_bytes_per_step is the average"},
            "gpu_launches": launches,
            "clocks": clk,
            "stats": stats,
            "fp64_path": fp64,
            "stat_error": stat_err,
            "speedup_vs_fp64": (value / fp64["value"]) if fp64 else None,
            "speedup_note": "the bench value over the FP64 path's rate, both over full runs from t = 0 to the "
                            "final time of the same levels (FP64 at M = 2 x stat_m)",
        }
        print(json.dumps(line), flush=True)
    ens.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=7)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--m", type=int, default=M_PER_GPU)
    ap.add_argument("--solver-steps", type=int, default=64,
                    help="fixed steps per bench step when --t-final is 0; the statistic-error check's horizon")
    ap.add_argument("--t-final", type=float, default=0.0035, help="the run's final time (0: fixed steps)")
    ap.add_argument("--dt-snap", type=float, default=0.0005, help="output interval: one bench step per output time")
    ap.add_argument("--stat-m", type=int, default=16,
                    help="realizations of the precision legs (FP64 path rate, statistic errors); 0: skip them")
    ap.add_argument("--cpu-steps", type=int, default=30)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
