"""Autotuner for the round kernel's launch knobs.

For each graph class it times the deterministic round kernel (CUDA events inside the library, on
the launching stream) over a grid of knobs -- the largest degree handled by one thread
(small_max_degree), the adjacency entries per warp work item (chunk), resident blocks per SM and
the compact sweep -- and writes the fastest setting per class to a JSON table.  `options_for(graph)`
returns the tuned gc_options for a graph from that table (library defaults when there is none).

Classes are decided from the degree sequence alone: "powerlaw" when the largest degree exceeds 50
times the average, else "uniform"; each is split into "small" (< 100,000 vertices) and "large".
Every entry records the digest of the library sources it was tuned on; an entry tuned on other
sources is stale and ignored (library defaults apply) until the tuner runs again.

    python -m paper_1509_08267_gb300.autotune [--out tuning.json] [--quick]
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import statistics

import numpy as np

from . import FLAG_FULL_SWEEP, FLAG_TIMING, Options, color, color_batch
from ._build import source_sha256

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")

GRID = {
    "small_max_degree": [32, 63, 127],
    "chunk": [256, 512, 1024],
    "blocks_per_sm": [0, 3],
    "compact": [False, True],
    "core_vertices": [0, -1],
}


def graph_class(n: int, degrees: np.ndarray) -> str:
    if n == 0:
        return "uniform-small"
    avg = max(float(degrees.mean()), 1e-9)
    shape = "powerlaw" if float(degrees.max()) > 50 * avg else "uniform"
    return f"{shape}-{'small' if n < 100_000 else 'large'}"


def _options(cfg: dict, timing: bool = True) -> Options:
    flags = (FLAG_TIMING if timing else 0) | (0 if cfg["compact"] else FLAG_FULL_SWEEP)
    return Options(small_max_degree=cfg["small_max_degree"], chunk=cfg["chunk"],
                   blocks_per_sm=cfg["blocks_per_sm"], flags=flags, core_vertices=cfg.get("core_vertices", 0))


def time_config(rowptr, colidx, cfg: dict, repeats: int = 3, seed: int = 7) -> float:
    """Median round-kernel milliseconds of deterministic coloring with the given knobs."""
    color(rowptr, colidx, "det", seed, options=_options(cfg))  # warm-up
    ms = [color(rowptr, colidx, "det", seed, options=_options(cfg)).stats.kernel_ms for _ in range(repeats)]
    return statistics.median(ms)


def time_config_batch(args, cfg: dict, repeats: int = 3, seed: int = 7) -> float:
    """Median round-kernel milliseconds of a deterministic batched coloring (args: the four packed
    arrays on the device)."""
    color_batch(*args, "det", seed, options=_options(cfg))
    ms = [color_batch(*args, "det", seed, options=_options(cfg), stats=True)[3].kernel_ms for _ in range(repeats)]
    return statistics.median(ms)


def tune(samples: dict, grid: dict = GRID, repeats: int = 3, log=print) -> dict:
    """samples: class name -> callable returning a timing function of a config."""
    table = {}
    keys = list(grid)
    for cls, timer in samples.items():
        best = None
        for values in itertools.product(*(grid[k] for k in keys)):
            cfg = dict(zip(keys, values))
            ms = timer(cfg)
            log(f"{cls:16s} {cfg} {ms:9.3f} ms")
            if best is None or ms < best[1]:
                best = (cfg, ms)
        table[cls] = {**best[0], "kernel_ms": best[1], "sources_sha256": source_sha256()}
    return table


def _entry(table_path: str, key: str) -> dict | None:
    """The table's entry `key` if it was tuned on the current sources."""
    try:
        with open(table_path) as f:
            entry = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    if not entry or entry.get("sources_sha256") != source_sha256():
        return None
    return entry


def options_for(n: int, degrees: np.ndarray, table_path: str = TABLE) -> Options:
    """Tuned options for a graph (library defaults if no current entry for its class)."""
    entry = _entry(table_path, graph_class(n, degrees))
    return _options(entry, timing=False) if entry else Options()


def options_for_graph(rowptr, table_path: str = TABLE) -> tuple[Options, str | None]:
    """options_for from a CSR row-offset array (numpy or a tensor); also returns the class name
    when a current entry was used, else None."""
    rp = rowptr.cpu().numpy() if hasattr(rowptr, "cpu") else np.asarray(rowptr)
    n = len(rp) - 1
    deg = np.diff(rp)
    cls = graph_class(n, deg)
    entry = _entry(table_path, cls)
    return (_options(entry, timing=False), cls) if entry else (Options(), None)


def batch_options(table_path: str = TABLE) -> Options:
    """Tuned options for gc_color_batch (the table's "batch" entry; library defaults without one)."""
    entry = _entry(table_path, "batch")
    return _options(entry, timing=False) if entry else Options()


def main():
    import torch

    import graphgen as gg

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--quick", action="store_true", help="one sample per class, fewer knobs")
    ap.add_argument("--batch-sample", default="batch256",
                    help="batch the 'batch' entry is tuned on: batchG = G mixed graphs (seed 3)")
    ap.add_argument("--only-batch", action="store_true", help="tune only the 'batch' entry (others kept)")
    args = ap.parse_args()
    dev = torch.device("cuda", 0)

    def on_device(g):
        return torch.from_numpy(g.rowptr).to(dev), torch.from_numpy(g.colidx).to(dev)

    grid = GRID if not args.quick else {"small_max_degree": [63, 127], "chunk": [512, 1024], "blocks_per_sm": [0],
                                        "compact": [False, True], "core_vertices": [0, -1]}
    table = {}
    if args.only_batch:
        try:
            with open(args.out) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    else:
        samples = {}
        for cls, make in [("powerlaw-large", lambda: gg.workload("rmat22")),
                          ("uniform-large", lambda: gg.stencil27(96)),
                          ("uniform-small", lambda: gg.workload("er10k")),
                          ("powerlaw-small", lambda: gg.rmat(16, 12, 5))]:
            g = make()
            rp, ci = on_device(g)
            samples[cls] = (lambda rp, ci: (lambda cfg: time_config(rp, ci, cfg)))(rp, ci)
        table = tune(samples, grid)
    b = gg.batch_mix(int(args.batch_sample[len("batch"):]), 3)
    bargs = [torch.from_numpy(a).to(dev) for a in (b.vtx_off, b.edge_off, b.rowptr, b.colidx)]
    bt = tune({"batch": lambda cfg: time_config_batch(bargs, cfg)}, grid)
    table.update(bt)
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print(json.dumps(table, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()
