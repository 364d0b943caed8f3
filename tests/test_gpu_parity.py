"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

FP64 path: <= 1e-12 per cell in the norms of tests/gpu_helpers.py over the
first 10 steps (the horizon over which round-off differences stay below that
level: the jet's shear layers amplify them ~10x every 5 steps).
"""

import numpy as np
import pytest
import torch

from oracle import oracle as O
from tests import gpu_helpers as H
from paper_2605_25282_gb300 import vlbm
from tests import inputs

pytestmark = pytest.mark.gpu

RTOL64 = 1e-12


def test_fp64_jet_smallest_config_10_steps():
    # 200 x 100, M = 4, seed 0, R-theta limiter: full fields after 10 steps.
    nx, ny, M = 200, 100, 4
    ref = H.oracle_jet(nx, ny, M, 10)
    ens = H.gpu_jet([(nx, ny)], M)
    ens.step(10)
    u, pops = ens.get_state(0)
    t, s = ens.time(0)
    u, pops = H.to_np(u), H.to_np(pops)
    assert np.all(s == 10)
    assert np.allclose(t, ref["t"], rtol=1e-14, atol=0)
    assert H.rel_err_cons(u, ref["u"]).max() <= RTOL64
    assert H.rel_err_pressure(u, ref["u"]).max() <= RTOL64
    assert H.rel_err_pops(pops, ref["pops"], ref["u"]).max() <= RTOL64
    # the solution moved: the jet entered the domain
    assert np.abs(u[:, 1, :, 1:4]).max() > 100.0


@pytest.mark.parametrize("limiter", [0])
def test_fp64_limiter_modes(limiter):
    # theta = 1 on the jet goes non-positive in the oracle itself (the unlimited
    # scheme at Mach 2000); it is covered on smooth data by the random-state test
    nx, ny, M = 96, 40, 2
    ref = H.oracle_jet(nx, ny, M, 8, limiter=limiter)
    ens = H.gpu_jet([(nx, ny)], M, limiter=limiter)
    ens.step(8)
    u, pops = map(H.to_np, ens.get_state(0))
    assert H.rel_err_cons(u, ref["u"]).max() <= RTOL64
    assert H.rel_err_pops(pops, ref["pops"], ref["u"]).max() <= RTOL64


def test_fp64_ragged_tiles_and_levels_in_one_launch():
    # interior extents that are not multiples of the tile or of the march's
    # strips, five levels at once, including single interior rows and columns
    levels = [(67, 29), (134, 58), (9, 3), (3, 7), (31, 5)]
    M, n = 3, 10
    ens = H.gpu_jet(levels, M)
    ens.step(n)
    for l, (nx, ny) in enumerate(levels):
        ref = H.oracle_jet(nx, ny, M, n)
        u, pops = map(H.to_np, ens.get_state(l))
        assert H.rel_err_cons(u, ref["u"]).max() <= RTOL64, l
        assert H.rel_err_pops(pops, ref["pops"], ref["u"]).max() <= RTOL64, l
        t, s = ens.time(l)
        assert np.allclose(t, ref["t"], rtol=1e-14, atol=0)


@pytest.mark.parametrize("design", [0, 1])
@pytest.mark.parametrize("limiter,rough", [(2, 0.3), (0, 0.3), (1, 0.0), (2, 0.0)])
def test_fp64_random_states(limiter, rough, design, monkeypatch):
    # both FP64 designs (0: tiles, 1: warp march, whose limiter queues the
    # divisions and roots of a row for the warp: on the rough states most
    # sides need both, more than one pass of 32); 45 columns are two strips
    monkeypatch.setenv("VLBM_F64_VARIANT", str(design))
    nx, ny, M = 45, 37, 2
    seed = 11
    g = O.Grid(nx, ny)
    P = H.oracle_params(limiter)
    ens = H.gpu_jet([(nx, ny)], M, limiter=limiter, seed=seed)
    us, ps = [], []
    for m in range(M):
        u, p = inputs.random_state(100 + m, nx, ny, rough=rough)
        us.append(u)
        ps.append(p)
    ens.set_state(torch.tensor(np.stack(us)), torch.tensor(np.stack(ps)))
    nsteps = 3
    ens.step(nsteps)
    assert ens.step_design()[0] == design
    ug, pg = map(H.to_np, ens.get_state(0))
    for m in range(M):
        inl = O.inlet(g, P, O.Jet(), seed, m)
        u, p = us[m], ps[m]
        for _ in range(nsteps):
            a = O.kinetic_speed(g, P, u)
            u, p, _ = O.step(g, P, a, u, p, inl, check=False)
        assert H.rel_err_cons(ug[m], u).max() <= RTOL64, m
        assert H.rel_err_pops(pg[m], p, u).max() <= RTOL64, m


def test_fp64_landing_on_output_time():
    nx, ny, M = 120, 60, 2
    t_end = 1.0e-4  # ~6 steps at this resolution, the last one landing
    ref = H.oracle_jet(nx, ny, M, 1000, t_end=t_end)
    ens = H.gpu_jet([(nx, ny)], M)
    ens.advance_to(t_end)
    t, s = ens.time(0)
    assert np.array_equal(s, ref["steps"])
    assert np.all(t == t_end)
    u = H.to_np(ens.get_state(0, pops=False)[0])
    assert H.rel_err_cons(u, ref["u"]).max() <= RTOL64
    # stepping on afterwards resumes from the landed state
    ens.step(1)
    t2, s2 = ens.time(0)
    assert np.all(s2 == s + 1) and np.all(t2 > t)


def test_fp64_moments_match_oracle():
    nx, ny, M = 80, 40, 2
    ref = H.oracle_jet(nx, ny, M, 10)
    ens = H.gpu_jet([(nx, ny)], M)
    ens.step(10)
    mo = {k: H.to_np(v) for k, v in ens.moments(0).items()}
    g = O.Grid(nx, ny)
    for m in range(M):
        rho, v1, v2, p = O.moments(g, H.oracle_params(), ref["u"][m])
        K = 0.5 * rho * (v1 ** 2 + v2 ** 2)
        assert np.abs(mo["rho"][m] - rho).max() <= RTOL64 * np.abs(rho).max()
        assert np.all(np.abs(mo["p"][m] - p) <= RTOL64 * (np.abs(p) + K))
        vs = np.sqrt(2 * K / rho) + np.sqrt(p / rho)
        assert np.all(np.abs(mo["u"][m] - v1) <= RTOL64 * vs)
        assert np.all(np.abs(mo["v"][m] - v2) <= RTOL64 * vs)
    dens = H.to_np(ens.density(0, f32=False))
    assert np.array_equal(dens, mo["rho"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nested_prefix_realizations(precision):
    # Sec. 3.1: nested sample sets are prefixes of the full ensemble
    a = H.gpu_jet([(64, 32)], 2, precision=precision)
    b = H.gpu_jet([(64, 32)], 5, precision=precision)
    a.step(12)
    b.step(12)
    ua, _ = a.get_state(0)
    ub, _ = b.get_state(0, 0, 2)
    assert torch.equal(ua, ub)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_save_load_resume_is_bit_identical(precision):
    ens = H.gpu_jet([(64, 32), (128, 64)], 3, precision=precision)
    ens.step(5)
    blob = ens.save()
    ens.step(7)
    ua = [ens.get_state(l)[0].clone() for l in range(2)]
    ta = ens.time(1)
    ens.load(blob)
    ens.step(7)
    for l in range(2):
        assert torch.equal(ens.get_state(l)[0], ua[l])
    tb = ens.time(1)
    assert np.array_equal(ta[0], tb[0]) and np.array_equal(ta[1], tb[1])


def test_fp64_positivity_over_smallest_config():
    # 200 x 100, M = 4, 500 steps: no realization raises a flag
    ens = H.gpu_jet([(200, 100)], 4)
    ens.step(500)
    ens.sync()
    t, s = ens.time(0)
    assert np.all(s == 500)
    mo = ens.moments(0)
    assert float(mo["rho"].min()) > 0 and float(mo["p"].min()) > 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_realization_block_init_equals_slice_of_full_ensemble(precision):
    # Sec. 3.1: realization m depends on (seed, m) only, so a block of
    # realizations m_begin .. m_begin + M - 1 initialised on its own (what each
    # rank of a multi-GPU run does) advances exactly like the same realizations
    # of the whole ensemble; two levels at once
    levels = [(64, 32), (128, 64)]
    blk = vlbm.Ensemble(levels, precision=precision, relax=H.relax())
    blk.init(0, 2, m_begin=3)
    full = H.gpu_jet(levels, 5, precision=precision)
    blk.step(12)
    full.step(12)
    for l in range(len(levels)):
        ub, _ = blk.get_state(l)
        uf, _ = full.get_state(l, 3, 2)
        assert torch.equal(ub, uf), l
        tb, sb = blk.time(l)
        tf, sf = full.time(l)
        assert np.array_equal(tb, tf[3:5]) and np.array_equal(sb, sf[3:5])
    if precision == "fp64":
        # and it is the oracle's realizations 3 and 4
        ref = H.oracle_jet(64, 32, 2, 12, m0=3)
        u = H.to_np(blk.get_state(0)[0])
        assert H.rel_err_cons(u, ref["u"]).max() <= RTOL64
