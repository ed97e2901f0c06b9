"""Partition mode (Algorithm 1 of Section 3.1 with p blocks of consecutive ids) on the GPU versus the
CPU oracle's literal rendition: bit-exact colors, color count, rounds and per-round worklist sizes
for several p; p = 1 is sequential First Fit in id order (natural-order greedy); Lemma 2 bounds the
rounds by p + 1."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def run_part(gc, g, p, stats=True):
    import torch
    rp = torch.from_numpy(np.ascontiguousarray(g.rowptr)).cuda()
    ci = torch.from_numpy(np.ascontiguousarray(g.colidx if g.nnz else np.zeros(0, np.int32))).cuda()
    r = gc.color(rp, ci, "partition", 0, options=gc.Options(partitions=p), stats=stats)
    return r


def assert_partition_parity(gc, g, p):
    ref = oracle.partition(g, p)
    assert ref.status == 0
    r = run_part(gc, g, p)
    np.testing.assert_array_equal(r.colors.cpu().numpy(), ref.colors, err_msg=f"{g.name} p={p}")
    assert (r.ncolors, r.rounds) == (ref.ncolors, ref.rounds)
    if g.n > 0:
        np.testing.assert_array_equal(r.stats.wl_size, ref.wl_size)
    assert r.rounds <= min(p, max(g.n, 1)) + 1  # Lemma 2
    return ref


GRAPHS = [
    lambda: gg.complete(1), lambda: gg.complete(40), lambda: gg.path(97), lambda: gg.cycle(1000),
    lambda: gg.star(5000), lambda: gg.crown(40), lambda: gg.empty(77), lambda: gg.grid5(37, 29),
    lambda: gg.stencil27(9), lambda: gg.er(3000, 12.0, 5), lambda: gg.rmat(12, 16, 2),
]


@pytest.mark.parametrize("make", GRAPHS)
@pytest.mark.parametrize("p", [1, 2, 7, 64, 4096])
def test_partition_matches_oracle(gclib, make, p):
    assert_partition_parity(gclib, make(), p)


def test_one_block_is_natural_greedy(gclib):
    # with a single block, phase 1 is sequential First Fit in id order and nothing conflicts
    g = gg.rmat(13, 8, 3)
    r = run_part(gclib, g, 1)
    colors, nc = oracle.greedy(g)
    np.testing.assert_array_equal(r.colors.cpu().numpy(), colors)
    assert (r.ncolors, r.rounds) == (nc, 1)


def test_one_block_per_vertex(gclib):
    # p = n: every vertex is its own block, and the vertex with the larger id keeps its color
    g = gg.er(2000, 8.0, 11)
    assert_partition_parity(gclib, g, g.n)


def test_default_partitions_proper(gclib):
    g = gg.rmat(16, 16, 4)
    r = run_part(gclib, g, 0, stats=False)
    c = r.colors.cpu().numpy()
    assert oracle.count_conflicts(g, c) == 0
    assert c.min() >= 0 and np.all(c <= g.degrees())
    assert r.ncolors == oracle.distinct_colors(c)


def test_partition_rejects_bad_entry(gclib):
    g = gg.path(10)
    ci = g.colidx.copy()
    ci[3] = 10  # out of range
    with pytest.raises(gclib.GCError) as e:
        gclib.color(g.rowptr, ci, "partition", 0, options=gclib.Options(partitions=3))
    assert e.value.status == gclib.GC_ERR_INVALID_GRAPH


def test_partition_batch_unsupported(gclib):
    b = gg.pack([gg.path(5), gg.path(7)])
    with pytest.raises(gclib.GCError) as e:
        gclib.color_batch(b.vtx_off, b.edge_off, b.rowptr, b.colidx, "partition", 0)
    assert e.value.status == gclib.GC_ERR_INVALID_ARG
