"""GPU statistics kernel (through stats_w1_mean_std) against the oracle's
restriction + mean / population std / one-point W1 (Sec. 3.2, Sec. 3.4).

Sums of M values in a different order differ by ~M eps: the bar is 1e-12
relative to the cell's scale (the sample magnitude).
"""

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2605_25282_gb300 import vlbm
from tests import inputs

pytestmark = pytest.mark.gpu


def run(a, b, f32=False):
    dt = torch.float32 if f32 else torch.float64
    ta = torch.tensor(a, dtype=dt, device="cuda")
    tb = torch.tensor(b, dtype=dt, device="cuda")
    out = vlbm.stats_w1_mean_std(ta, tb)
    torch.cuda.synchronize()
    if f32:
        a = ta.double().cpu().numpy()
        b = tb.double().cpu().numpy()
    ref = O.stats_w1_mean_std(a, b)
    return {k: v.cpu().numpy() for k, v in out.items()}, ref, a


@pytest.mark.parametrize("M", [1, 2, 7, 64, 1000, 4096])
@pytest.mark.parametrize("r", [1, 2])
def test_stats_match_oracle(M, r):
    ny, nx = (13, 7) if M < 1000 else (4, 6)
    a = inputs.random_samples(1, M, ny, nx)
    b = inputs.random_samples(2, M, r * ny, r * nx)
    got, ref, _ = run(a, b)
    scale = np.abs(a).max()
    for key, rv in zip(("mean_a", "std_a", "mean_b", "std_b", "w1"), ref):
        assert np.abs(got[key] - rv).max() <= 1e-12 * scale, key


@pytest.mark.parametrize("dist", ["lognormal", "ties"])
def test_stats_fp32_inputs_and_ties(dist):
    a = inputs.random_samples(3, 33, 5, 9, dist)
    b = inputs.random_samples(4, 33, 20, 36, dist)
    got, ref, a64 = run(a, b, f32=True)
    scale = np.abs(a64).max()
    for key, rv in zip(("mean_a", "std_a", "mean_b", "std_b", "w1"), ref):
        assert np.abs(got[key] - rv).max() <= 1e-12 * scale, key


def test_stats_identical_ensembles_and_shift():
    a = inputs.random_samples(5, 100, 6, 6)
    got, _, _ = run(a, a)
    assert np.all(got["w1"] == 0) and np.array_equal(got["mean_a"], got["mean_b"])
    got, _, _ = run(a, a + 0.5)
    assert np.allclose(got["w1"], 0.5, rtol=1e-12)


@pytest.mark.parametrize("r, f32_in, f32_out", [(1, False, False), (2, True, False), (8, False, True), (5, True, True)])
def test_restrict_matches_oracle(r, f32_in, f32_out):
    # the restriction operator R of Sec. 3.3 (block average, same summation order)
    M, nyc, nxc = 3, 7, 11
    rng = np.random.default_rng(r)
    fine = rng.lognormal(0.0, 0.5, (M, nyc * r, nxc * r))
    if f32_in:
        fine = fine.astype(np.float32)
    got = vlbm.stats_restrict(torch.from_numpy(fine).cuda(), r, f32=f32_out)
    want = O.restrict(fine.astype(np.float64), r)
    if f32_out:
        assert np.array_equal(got.cpu().numpy(), want.astype(np.float32))
    else:
        assert np.array_equal(got.cpu().numpy(), want)


def test_sharded_statistics_single_process_equal_direct():
    # the multi-process statistics path on one NCCL rank equals the direct call
    import os
    import socket

    import torch.distributed as dist

    from paper_2605_25282_gb300 import sharded

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        rng = np.random.default_rng(5)
        a = torch.from_numpy(rng.lognormal(0, 0.3, (9, 10, 12)).astype(np.float32)).cuda()
        b = torch.from_numpy(rng.lognormal(0, 0.3, (9, 20, 24)).astype(np.float32)).cuda()
        got = sharded.gpu_statistics(a, b)
        want = vlbm.stats_w1_mean_std(a, b)
        for k in want:
            assert torch.equal(got[k], want[k]), k
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("M, r, npd, f32", [(7, 1, 3, False), (64, 2, 4, True), (33, 3, 2, False), (1, 1, 2, False)])
def test_two_point_w1_matches_oracle(M, r, npd, f32):
    # Eq. (w2): exact optimal assignment per point pair against scipy's
    rng = np.random.default_rng(M + r)
    ny, nx = 9, 11
    a = rng.lognormal(0.0, 0.5, (M, ny, nx))
    b = rng.lognormal(0.1, 0.4, (M, ny * r, nx * r))
    if f32:
        a, b = a.astype(np.float32), b.astype(np.float32)
    w, pairs = vlbm.stats_w1_two_point(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), npd)
    want, want_pairs = O.w1_two_point(a.astype(np.float64), b.astype(np.float64), npd)
    assert np.allclose(pairs.cpu().numpy(), want_pairs, rtol=1e-12, atol=1e-15)
    assert abs(float(w) - want) <= 1e-12 * want


def test_two_point_w1_identities():
    rng = np.random.default_rng(2)
    a = torch.from_numpy(rng.lognormal(size=(20, 8, 8))).cuda()
    w, pairs = vlbm.stats_w1_two_point(a, a, 4)
    assert float(w) == 0.0
    # a translated copy: every joint law moves by (0.1, 0.1)
    w, pairs = vlbm.stats_w1_two_point(a, a + 0.1, 4)
    assert torch.allclose(pairs, torch.full_like(pairs, 0.1 * np.sqrt(2.0)), rtol=1e-12)


def test_statistics_on_another_stream_are_ordered_with_the_callers():
    # inputs written on the caller's stream just before the call and results
    # copied there just after, while the call runs on another stream: the
    # binding orders both ways, so the copies equal a call on the caller's
    # own stream after a synchronization
    M, ny, nx = 256, 200, 300
    side = torch.cuda.Stream()
    g = torch.Generator(device="cuda").manual_seed(3)
    base = torch.rand((M, ny, nx), device="cuda", dtype=torch.float64, generator=g) + 0.5
    torch.cuda.synchronize()
    for _ in range(3):
        a = torch.exp(torch.log(base))  # queued on the caller's stream
        b = torch.exp(torch.log(base.flip(0) * 1.1))
        got = {k: v.clone() for k, v in vlbm.stats_w1_mean_std(a, b, stream=side).items()}
        torch.cuda.synchronize()
        ref = vlbm.stats_w1_mean_std(a, b)
        torch.cuda.synchronize()
        for k in ("mean_a", "std_a", "mean_b", "std_b", "w1"):
            assert torch.equal(got[k], ref[k]), k
