"""Ensemble statistics of the mixed path against the oracle's FP64 ensemble
(Sec. 3.2, Eqs. (mean), (std), (w1disc)) on the 200 x 100 Mach 2000 jet,
seed 0, M = 32 realizations on both sides.

Norm, L1 over the domain like the paper's functionals (Sec. 3.4):
sum |s_gpu - s_orc| / sum |s_orc| for the per-cell mean and std of rho, and
the per-cell one-point W1 between the two ensembles over sum |mean_orc|.

Short horizon (64 steps): the realizations still follow each other, and every
statistic agrees to 1e-3.

Long horizon (500 steps, t ~ 0.0037, the jet's final time on this grid):
the realizations have diverged pathwise.  Even the GPU's FP64 path, which
equals the oracle to round-off per step (1e-12 per cell over 10 steps, 1e-9
after 64), is then ~1e-2 away from it (4e-2 for the std), and no precision
reproduces a given ensemble to 1e-3.  What an ensemble of M realizations can be asked is
to estimate the statistics as well as any other ensemble of M realizations:
the bar is the Monte-Carlo error at matched M, the distance between the
oracle's ensemble and independent oracle ensembles of the same size
(realizations M .. 2M - 1, 2M .. 3M - 1, ...).  Once a statistic has fully
decorrelated (the std does first) the mixed path's distance is one more draw
of that same distance, so the bar is its mean over four independent
ensembles plus three times their spread, for every statistic.
"""

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_25282_gb300 import vlbm

pytestmark = pytest.mark.gpu

NX, NY, M = 200, 100, 32
N_INDEPENDENT = 4


def _oracle_density(args):
    m, n, amp_change = args
    from oracle import oracle as Ow

    jet = Ow.Jet()
    if amp_change:
        jet = Ow.Jet(amp=jet.amplitudes() * (1.0 + amp_change))
    r = Ow.run_jet(Ow.Grid(NX, NY), Ow.Params(), jet, 0, m, 1, n, want_pops=False)
    return r["u"][0, 0]


@pytest.fixture(scope="module")
def oracle_runs():
    # one process per realization (spawn: this process already holds a CUDA context)
    with cf.ProcessPoolExecutor(os.cpu_count() or 1, mp_context=mp.get_context("spawn")) as ex:
        short = np.stack(list(ex.map(_oracle_density, [(m, 64, 0.0) for m in range(M)])))
        d = np.stack(list(ex.map(_oracle_density, [(m, 500, 0.0) for m in range((1 + N_INDEPENDENT) * M)])))
        control = np.stack(list(ex.map(_oracle_density, [(m, 500, 1e-7) for m in range(M)])))
    return {64: (short, None, None),
            500: (d[:M], [d[(i + 1) * M:(i + 2) * M] for i in range(N_INDEPENDENT)], control)}


def _errors(a, b):
    ma, sa, mb, sb, w1 = O.stats_w1_mean_std(a, b)
    return {"mean": np.abs(ma - mb).sum() / np.abs(mb).sum(), "std": np.abs(sa - sb).sum() / np.abs(sb).sum(),
            "w1": w1.sum() / np.abs(mb).sum()}


def _gpu_density(precision, n):
    ens = vlbm.Ensemble([(NX, NY)], precision=precision)
    ens.init(0, M)
    ens.step(n)
    ens.sync()
    d = ens.density(0, f32=False).cpu().numpy()
    ens.close()
    return d


def test_mixed_statistics_short_horizon_within_1e3(oracle_runs):
    ref, _, _ = oracle_runs[64]
    e = _errors(_gpu_density("mixed", 64), ref)
    print("mixed vs oracle, 64 steps:", e)
    assert max(e.values()) <= 1e-3, e


def test_mixed_statistics_long_horizon_within_monte_carlo_error(oracle_runs):
    ref, independent, control = oracle_runs[500]
    mc = [_errors(x, ref) for x in independent]
    mixed = _errors(_gpu_density("mixed", 500), ref)
    fp64 = _errors(_gpu_density("fp64", 500), ref)
    ctl = _errors(control, ref)
    print("500 steps: mixed vs oracle", mixed, "| FP64 path vs oracle", fp64,
          "| oracle with amplitudes x (1 + 1e-7) vs oracle", ctl, "| independent ensembles vs oracle", mc)
    for k in ("mean", "std", "w1"):
        d = np.array([e[k] for e in mc])
        bar = d.mean() + 3.0 * d.std(ddof=1)
        assert mixed[k] <= bar, (k, mixed[k], d)
        assert fp64[k] <= bar, (k, fp64[k], d)
