"""The multi-process path on CPU: two gloo ranks, each owning a realization
block, compute the ensemble statistics of Sec. 3.4 over both blocks through
the row-block all-to-all of paper_2605_25282_gb300.sharded.  The per-block
statistics and the restriction are the oracle's; the result must equal the
oracle's statistics of the whole ensemble exactly (the exchange only moves
samples, and realizations keep their global order)."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O

M_LOCAL, NY, NX, R = 5, 7, 6, 2


def block(rank, M):
    """Densities of the global realizations rank*M .. rank*M+M-1 (seeded by the global index)."""
    a, b = [], []
    for g in range(rank * M, rank * M + M):
        rng = np.random.default_rng(1000 + g)
        a.append(rng.lognormal(0.0, 0.4, (NY, NX)))
        b.append(rng.lognormal(0.0, 0.4, (R * NY, R * NX)))
    return np.array(a), np.array(b)


def oracle_stats(a, b):
    ma, sa, mb, sb, w1 = O.ensemble_stats(a.numpy(), b.numpy())
    return {k: torch.from_numpy(v) for k, v in zip(("mean_a", "std_a", "mean_b", "std_b", "w1"), (ma, sa, mb, sb, w1))}


def worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2605_25282_gb300 import sharded

        a, b = block(rank, M_LOCAL)
        got = sharded.sharded_statistics(torch.from_numpy(a), torch.from_numpy(b), oracle_stats,
                                         lambda x, r: torch.from_numpy(O.restrict(x.numpy(), r)))
        q.put((rank, {k: v.numpy() for k, v in got.items()}))
    finally:
        dist.destroy_process_group()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_statistics_equal_whole_ensemble(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    blocks = [block(r, M_LOCAL) for r in range(world)]
    A = np.concatenate([x[0] for x in blocks])
    B = np.concatenate([x[1] for x in blocks])
    want = dict(zip(("mean_a", "std_a", "mean_b", "std_b", "w1"), O.stats_w1_mean_std(A, B)))
    for r in range(world):
        for k, v in want.items():
            assert np.array_equal(results[r][k], v), (r, k)


def test_row_blocks_cover_rows():
    from paper_2605_25282_gb300 import sharded

    for ny in (1, 2, 7, 200, 401):
        for n in (1, 2, 3, 8):
            bl = sharded.row_blocks(ny, n)
            assert bl[0][0] == 0 and bl[-1][1] == ny
            assert all(bl[i][1] == bl[i + 1][0] for i in range(n - 1))
            assert max(b - a for a, b in bl) - min(b - a for a, b in bl) <= 1
