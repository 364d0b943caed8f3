"""Ensemble statistics over realization blocks held by several processes.

Stepping shards by realization with no exchange: process r owns the global
realizations [r M, (r + 1) M) (vlbm_init_ensemble_block; Philox counters are
global indices, Sec. 3.1).  The statistics of Sec. 3.4 need all N M samples of
a cell in one place (W1 sorts them), so they take one exchange: every process
restricts its fine level onto the coarse grid (Sec. 3.3), cuts the coarse grid
into N row blocks, and an all-to-all sends row block k of every local
realization to process k.  Process k then holds its rows for all realizations
in global order, computes mean / std / W1 there, and an all-gather assembles
the fields on every process.

The per-block statistics and the restriction are passed in as callables (the
library's kernels on GPUs; any implementation of the same definitions in a
CPU test), and the exchange runs on the given process group (NCCL or gloo).
"""

from __future__ import annotations

from typing import Callable

import torch
import torch.distributed as dist

StatsFn = Callable[[torch.Tensor, torch.Tensor], dict]
RestrictFn = Callable[[torch.Tensor, int], torch.Tensor]

FIELDS = ("mean_a", "std_a", "mean_b", "std_b", "w1")


def row_blocks(ny: int, n: int) -> list[tuple[int, int]]:
    """Rows [begin, end) of each of n blocks: sizes differ by at most one."""
    base, extra = divmod(ny, n)
    out, r = [], 0
    for k in range(n):
        h = base + (1 if k < extra else 0)
        out.append((r, r + h))
        r += h
    return out


def exchange_rows(local: torch.Tensor, group=None) -> torch.Tensor:
    """All-to-all of row blocks: local [M_local, ny, nx] -> [N * M_local, rows_k, nx]
    holding this process's row block k for every realization, in global order
    (process-major, which is the global index order of the realization blocks)."""
    n = dist.get_world_size(group)
    k = dist.get_rank(group)
    M, ny, nx = local.shape
    blocks = row_blocks(ny, n)
    h = max(b - a for a, b in blocks)
    # equal-size messages: every block padded to h rows
    send = torch.zeros((n, M, h, nx), dtype=local.dtype, device=local.device)
    for j, (a, b) in enumerate(blocks):
        send[j, :, : b - a] = local[:, a:b]
    recv = torch.empty_like(send)
    dist.all_to_all_single(recv, send, group=group)
    a, b = blocks[k]
    return recv[:, :, : b - a].reshape(n * M, b - a, nx).contiguous()


def sharded_statistics(dens_a: torch.Tensor, dens_b: torch.Tensor, stats_fn: StatsFn, restrict_fn: RestrictFn,
                       group=None) -> dict:
    """mean / std of both levels and one-point W1 over the realizations of all
    processes.  dens_a [M_local, ny, nx] (coarse level), dens_b
    [M_local, r ny, r nx] (fine level); the same M_local on every process.
    Returns full [ny, nx] FP64 fields on every process."""
    n = dist.get_world_size(group)
    M, ny, nx = dens_a.shape
    r = dens_b.shape[2] // nx
    if dens_b.shape[0] != M or dens_b.shape[1] != r * ny or dens_b.shape[2] != r * nx:
        raise ValueError("the fine level must be an integer refinement of the coarse level")
    mcount = torch.tensor([M], device=dens_a.device)
    mall = [torch.zeros_like(mcount) for _ in range(n)]
    dist.all_gather(mall, mcount, group=group)
    if any(int(x) != M for x in mall):
        raise ValueError("every process must hold the same number of realizations")
    fine = restrict_fn(dens_b, r) if r > 1 else dens_b
    a_rows = exchange_rows(dens_a, group)
    b_rows = exchange_rows(fine, group)
    blocks = row_blocks(ny, n)
    h = max(b - a for a, b in blocks)
    part = stats_fn(a_rows, b_rows) if a_rows.shape[1] > 0 else None
    out = {}
    for f in FIELDS:
        mine = torch.zeros((h, nx), dtype=torch.float64, device=dens_a.device)
        if part is not None:
            mine[: part[f].shape[0]] = part[f]
        gathered = [torch.empty_like(mine) for _ in range(n)]
        dist.all_gather(gathered, mine, group=group)
        out[f] = torch.cat([g[: b - a] for g, (a, b) in zip(gathered, blocks)], 0)
    return out


def gpu_statistics(dens_a: torch.Tensor, dens_b: torch.Tensor, group=None) -> dict:
    """sharded_statistics with the library's kernels (device tensors)."""
    from . import vlbm

    return sharded_statistics(dens_a, dens_b, lambda a, b: vlbm.stats_w1_mean_std(a, b),
                              lambda x, r: vlbm.stats_restrict(x, r), group)
