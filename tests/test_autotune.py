"""Host logic of the autotuner (no GPU): graph classes, table lookup and the grid search."""
import json

import numpy as np

import graphgen as gg
from paper_1509_08267_gb300 import FLAG_FULL_SWEEP, autotune


def test_graph_classes():
    g = gg.rmat(12, 16, 2)
    assert autotune.graph_class(g.n, g.degrees()) == "powerlaw-small"
    s = gg.stencil27(8)
    assert autotune.graph_class(s.n, s.degrees()) == "uniform-small"
    assert autotune.graph_class(200_000, np.full(200_000, 5)) == "uniform-large"


def test_options_lookup(tmp_path):
    sha = autotune.source_sha256()
    table = {"powerlaw-small": {"small_max_degree": 63, "chunk": 512, "blocks_per_sm": 3, "compact": True,
                                "kernel_ms": 1.0, "sources_sha256": sha},
             "batch": {"small_max_degree": 127, "chunk": 1024, "blocks_per_sm": 0, "compact": False,
                       "kernel_ms": 2.0, "sources_sha256": sha, "core_vertices": -1}}
    path = tmp_path / "t.json"
    path.write_text(json.dumps(table))
    g = gg.rmat(12, 16, 2)
    o = autotune.options_for(g.n, g.degrees(), str(path))
    assert (o.small_max_degree, o.chunk, o.blocks_per_sm) == (63, 512, 3) and not o.flags & FLAG_FULL_SWEEP
    s = gg.stencil27(8)
    assert autotune.options_for(s.n, s.degrees(), str(path)).chunk == 0  # no entry: library defaults
    assert autotune.batch_options(str(path)).chunk == 1024
    assert autotune.batch_options(str(path)).core_vertices == -1
    o2, cls = autotune.options_for_graph(g.rowptr, str(path))
    assert cls == "powerlaw-small" and o2.chunk == 512


def test_stale_entries_are_ignored(tmp_path):
    # an entry tuned on other sources does not apply: library defaults instead
    table = {"batch": {"small_max_degree": 63, "chunk": 256, "blocks_per_sm": 3, "compact": True, "kernel_ms": 1.0,
                       "sources_sha256": "0" * 64}}
    path = tmp_path / "t.json"
    path.write_text(json.dumps(table))
    assert autotune.batch_options(str(path)).chunk == 0
    assert autotune.options_for(1, np.zeros(1), str(tmp_path / "missing.json")).chunk == 0


def test_grid_search_picks_fastest():
    seen = []

    def timer(cfg):
        seen.append(cfg)
        return abs(cfg["chunk"] - 512) + (0 if cfg["compact"] else 1) + cfg["small_max_degree"] / 1000

    grid = {"small_max_degree": [32, 127], "chunk": [256, 512, 1024], "blocks_per_sm": [0], "compact": [False, True]}
    table = autotune.tune({"x": timer}, grid, log=lambda *_: None)
    assert len(seen) == 12
    best = table["x"]
    assert (best["chunk"], best["compact"], best["small_max_degree"]) == (512, True, 32)
    assert best["sources_sha256"] == autotune.source_sha256()
