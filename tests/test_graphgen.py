"""The seeded generators produce undirected simple graphs of the stated shapes (no GPU)."""
import numpy as np
import pytest

import graphgen as gg


def check_simple(g):
    rp, ci = g.rowptr, g.colidx
    assert rp[0] == 0 and rp[-1] == len(ci) and np.all(np.diff(rp) >= 0)
    if g.nnz == 0:
        return
    assert ci.min() >= 0 and ci.max() < g.n
    src = np.repeat(np.arange(g.n), np.diff(rp))
    assert not np.any(src == ci), "self-loop"
    # rows strictly increasing (sorted, no duplicates)
    same_row = src[1:] == src[:-1]
    assert np.all(ci[1:][same_row] > ci[:-1][same_row])
    # symmetric
    fwd = np.sort(src.astype(np.int64) * g.n + ci)
    rev = np.sort(ci.astype(np.int64) * g.n + src)
    assert np.array_equal(fwd, rev)


@pytest.mark.parametrize("make", [
    lambda: gg.er(1000, 8, 1), lambda: gg.er(2, 1, 3), lambda: gg.rmat(10, 16, 2), lambda: gg.rmat(11, 9.5, 4, n=1500),
    lambda: gg.stencil27(5), lambda: gg.grid5(6, 4), lambda: gg.complete(6), lambda: gg.crown(5),
    lambda: gg.star(9), lambda: gg.cycle(7), lambda: gg.path(1), lambda: gg.empty(3),
])
def test_simple_graphs(make):
    check_simple(make())


def test_stencil_counts():
    for L in (1, 2, 3, 7):
        g = gg.stencil27(L)
        assert g.nnz == (3 * L - 2) ** 3 - L ** 3
        if L >= 3:
            assert g.degrees().max() == 26 and g.degrees().min() == 7
    assert gg._L().gg_stencil27_nnz(256) == 432_677_880


def test_grid_counts():
    g = gg.grid5(10, 7)
    assert g.nnz == 2 * (9 * 7 + 10 * 6)


def test_er_pairs_and_determinism():
    a = gg.er(10_000, 16, 1)
    b = gg.er(10_000, 16, 1)
    assert np.array_equal(a.colidx, b.colidx)
    # 80,000 drawn pairs, a few duplicates removed
    assert 2 * 79_000 < a.nnz <= 2 * 80_000
    assert not np.array_equal(gg.er(10_000, 16, 2).colidx[:100], a.colidx[:100])


def test_rmat_skew_and_permutation():
    g = gg.rmat(14, 16, 2)
    d = g.degrees()
    assert d.max() > 50 * np.median(d[d > 0])  # power-law hubs
    p = gg.permutation(1000, 5)
    assert np.array_equal(np.sort(p), np.arange(1000))


def test_batch_pack_roundtrip():
    gs = [gg.complete(3), gg.empty(0), gg.er(50, 4, 2), gg.cycle(4)]
    b = gg.pack(gs)
    assert b.G == 4 and b.vtx_off[-1] == sum(g.n for g in gs) and b.edge_off[-1] == sum(g.nnz for g in gs)
    for i, g in enumerate(gs):
        h = b.graph(i)
        assert h.n == g.n and np.array_equal(h.rowptr, g.rowptr) and np.array_equal(h.colidx, g.colidx)


def test_batch_specs_distribution():
    specs = gg.batch_specs(4096, 3)
    ns = np.array([s.n for s in specs])
    assert ns.min() >= 100 and ns.max() <= 200_000
    assert 20_000 < ns.mean() < 33_000  # log-uniform on [100, 2e5] has mean ~26,300
    assert sum(s.kind == "er" for s in specs) == 2048
    er_d = [s.param for s in specs if s.kind == "er"]
    assert 4 <= min(er_d) and max(er_d) <= 64


def test_parallel_batch_generation_matches_graph_by_graph():
    fast = gg.batch_mix(30, 3, nmin=100, nmax=30_000)
    slow = gg.pack([gg.make_from_spec(s) for s in gg.batch_specs(30, 3, nmin=100, nmax=30_000)])
    for a, b in [(fast.vtx_off, slow.vtx_off), (fast.edge_off, slow.edge_off), (fast.rowptr, slow.rowptr),
                 (fast.colidx, slow.colidx)]:
        assert np.array_equal(a, b)
    for g in range(fast.G):
        check_simple(fast.graph(g))
