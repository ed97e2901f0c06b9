"""Coloring across several processes (one per GPU).

Two splits, both taken from the method itself:

* Graph-sharded batches (``shard_graphs``): a batch's graphs are independent problems, so each rank
  colors its own subset with ``color_batch``; nothing is exchanged.
* Vertex blocks of one graph (``color_blocks``): Algorithm 1 (Section 3.1) partitions V into blocks
  V_1..V_p of consecutive ids, one per thread.  Here one block per rank: every round each rank runs
  ``det_round`` over its block's worklist vertices, reading the colors as the round began, then the
  ranks exchange the new colors of the vertices that lost (the boundary vertices' colors are what
  the other blocks read next round).  Because the deterministic mode's rounds read only C_r and the
  priority key is global, the colors and the round count equal those of ``color`` for any number of
  blocks.

The rank's kernel and the exchange are passed in, so the same driver runs the library's round on
a GPU with NCCL, an in-process emulation of several blocks, or a plain CPU step under gloo in tests.
"""
from __future__ import annotations

import torch


def block_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Block `rank` of `world` over n vertices: ids [floor(rank n / world), floor((rank + 1) n / world))."""
    return n * rank // world, n * (rank + 1) // world


def shard_graphs(sizes, world: int) -> list[int]:
    """Owner rank of each graph of a batch: greedy by size (largest first onto the least loaded
    rank, ties to the lower rank), so the ranks' loads differ by at most one graph's size."""
    load = [0] * world
    owner = [0] * len(sizes)
    for g in sorted(range(len(sizes)), key=lambda g: (-int(sizes[g]), g)):
        r = min(range(world), key=lambda k: (load[k], k))
        owner[g] = r
        load[r] += int(sizes[g])
    return owner


def _initial_worklist(rowptr: torch.Tensor, lo: int, hi: int) -> torch.Tensor:
    # W_1 = the block's vertices with neighbours (an isolated vertex takes color 0 and is final)
    deg = rowptr[lo + 1: hi + 1] - rowptr[lo:hi]
    return torch.arange(lo, hi, dtype=torch.int32, device=rowptr.device)[deg > 0]


def color_blocks(rowptr: torch.Tensor, colidx: torch.Tensor, seed: int, step, exchange, rank: int = 0, world: int = 1,
                 max_rounds: int | None = None):
    """Deterministic coloring with vertex block `rank` of `world` on this process.

    step(colors_cur, worklist) -> (colors_next, lost): one round over the block's worklist (for
    example ``det_round`` on this rank's GPU).  exchange(ids, colors) -> (ids, colors): the losers'
    new colors of every rank (an all-gather).  Returns (colors of every vertex, rounds); every rank
    ends with the same colors."""
    n = rowptr.numel() - 1
    colors = torch.zeros(max(n, 0), dtype=torch.int32, device=rowptr.device)  # C_1 = 0 everywhere
    if n == 0:
        return colors, 0
    lo, hi = block_range(n, rank, world)
    work = _initial_worklist(rowptr, lo, hi)
    cap = max_rounds if max_rounds is not None else n + 1
    rounds = 0
    while True:
        if rounds >= cap:
            raise RuntimeError(f"worklist not empty after {rounds} rounds")
        rounds += 1
        nxt, lost = step(colors, work)
        m = lost != 0
        ids, cols = work[m], nxt[m]
        all_ids, all_cols = exchange(ids, cols)
        if all_ids.numel() == 0:
            return colors, rounds
        colors[all_ids.long()] = all_cols
        work = ids


def color_blocks_inprocess(rowptr: torch.Tensor, colidx: torch.Tensor, seed: int, step, world: int,
                           max_rounds: int | None = None):
    """The same rounds with all `world` blocks in this process, one after another each round (the
    exchange is a concatenation).  Returns (colors, rounds)."""
    n = rowptr.numel() - 1
    colors = torch.zeros(max(n, 0), dtype=torch.int32, device=rowptr.device)
    if n == 0:
        return colors, 0
    works = [_initial_worklist(rowptr, *block_range(n, r, world)) for r in range(world)]
    cap = max_rounds if max_rounds is not None else n + 1
    rounds = 0
    while True:
        if rounds >= cap:
            raise RuntimeError(f"worklist not empty after {rounds} rounds")
        rounds += 1
        changes = []
        for r in range(world):
            nxt, lost = step(colors, works[r])
            m = lost != 0
            works[r] = works[r][m]
            changes.append((works[r], nxt[m]))
        ids = torch.cat([c[0] for c in changes])
        if ids.numel() == 0:
            return colors, rounds
        colors[ids.long()] = torch.cat([c[1] for c in changes])


def allgather_exchange(group=None):
    """exchange() for color_blocks over torch.distributed (gloo or NCCL): an all-gather of each
    rank's (ids, colors), padded to the largest rank's count."""
    import torch.distributed as dist

    def exchange(ids: torch.Tensor, cols: torch.Tensor):
        world = dist.get_world_size(group)
        cnt = torch.tensor([ids.numel()], dtype=torch.int64, device=ids.device)
        cnts = [torch.zeros_like(cnt) for _ in range(world)]
        dist.all_gather(cnts, cnt, group=group)
        sizes = [int(c.item()) for c in cnts]
        top = max(sizes)
        if top == 0:
            return ids[:0], cols[:0]
        pad = torch.zeros(2, top, dtype=torch.int32, device=ids.device)
        pad[0, : ids.numel()] = ids
        pad[1, : cols.numel()] = cols
        bufs = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(bufs, pad, group=group)
        got_ids = torch.cat([b[0, :k] for b, k in zip(bufs, sizes)])
        got_cols = torch.cat([b[1, :k] for b, k in zip(bufs, sizes)])
        return got_ids, got_cols

    return exchange


def gpu_step(rowptr: torch.Tensor, colidx: torch.Tensor, seed: int):
    """step() for color_blocks: the library's round (gc_det_round) on the tensors' GPU."""
    from . import det_round

    def step(colors, work):
        if work.numel() == 0:
            z = work[:0]
            return z, z
        return det_round(rowptr, colidx, seed, colors, work)

    return step
