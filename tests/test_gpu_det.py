"""Deterministic mode on the GPU versus the CPU oracle: bit-exact colors, color count, round count and
per-round worklist statistics (Algorithm 1, Section 3.1, with the hash-priority reading)."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _dev(g):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(g.rowptr)).cuda(),
            torch.from_numpy(np.ascontiguousarray(g.colidx if g.nnz else np.zeros(0, np.int32))).cuda())


def run_det(gc, g, seed, options=None, stats=False):
    rp, ci = _dev(g)
    r = gc.color(rp, ci, "det", seed, options=options, stats=stats)
    return r.colors.cpu().numpy(), r.ncolors, r.rounds, r.stats


def core_variants(gc, g):
    """The library default (small graphs run round 1 in the shared-memory core phase and the rest
    in the cluster's tail phase), the regular round kernel alone, the core phase without the tail,
    and hand-overs part-way through the run: to the core by a vertex cap and by an entry cap (which
    makes the rounds count their worklists' entries), and from the core to the tail."""
    out = [gc.Options(), gc.Options(core_vertices=-1), gc.Options(tail_vertices=-1), gc.Options(tail_vertices=4096)]
    for cap in (max(1, g.n // 10), max(1, g.n // 3)):
        out.append(gc.Options(core_vertices=cap))
    if g.nnz > 8:
        out.append(gc.Options(core_entries=max(1, g.nnz // 8)))
    out.append(gc.Options(core_vertices=max(1, g.n // 3), tail_vertices=max(1, g.n // 20)))
    return out


def assert_parity(gc, g, seed, options=None, check_stats=True):
    ref = oracle.det(g, seed)
    assert ref.status == 0
    for opt in ([options] if options is not None else core_variants(gc, g)):
        colors, nc, rounds, st = run_det(gc, g, seed, options=opt, stats=check_stats)
        np.testing.assert_array_equal(colors, ref.colors, err_msg=f"{g.name} seed {seed} {opt}")
        assert nc == ref.ncolors, opt
        assert rounds == ref.rounds, opt
        if check_stats and g.n > 0:
            np.testing.assert_array_equal(st.wl_size, ref.wl_size, err_msg=str(opt))
            np.testing.assert_array_equal(st.wl_degsum, ref.wl_degsum, err_msg=str(opt))
    return ref


SPECIAL = [
    lambda: gg.complete(1), lambda: gg.complete(2), lambda: gg.complete(5), lambda: gg.complete(33),
    lambda: gg.complete(40), lambda: gg.complete(200), lambda: gg.path(2), lambda: gg.path(97),
    lambda: gg.cycle(3), lambda: gg.cycle(1000), lambda: gg.star(31), lambda: gg.star(32),
    lambda: gg.star(5000), lambda: gg.crown(40), lambda: gg.crown(40, interleaved=False), lambda: gg.empty(1),
    lambda: gg.empty(77), lambda: gg.grid5(7, 9), lambda: gg.stencil27(4), lambda: gg.stencil27(9),
]


@pytest.mark.parametrize("make", SPECIAL)
@pytest.mark.parametrize("seed", [0, 7])
def test_special_graphs(gclib, make, seed):
    assert_parity(gclib, make(), seed)


def test_er10k_seed7(gclib):
    # Erdos-Renyi n=10,000, average degree 16, edges from seed 1, hash seed 7
    assert_parity(gclib, gg.workload("er10k"), 7)


@pytest.mark.parametrize("scale", [8, 12, 15])
@pytest.mark.parametrize("seed", [1, 7, 2**63 + 5])
def test_rmat_small(gclib, scale, seed):
    assert_parity(gclib, gg.rmat(scale, 16, 2), seed)


def test_ragged_er(gclib):
    for n, d in [(31, 3.0), (33, 5.0), (777, 9.0), (4099, 40.0)]:
        assert_parity(gclib, gg.er(n, d, 11), 3)


def test_isolated_mixed(gclib):
    # graph with isolated vertices interleaved with a dense core
    edges = [(i, j) for i in range(0, 60, 2) for j in range(i + 2, 60, 2)]
    assert_parity(gclib, gg.from_edges(61, edges), 5)


def test_window_rescan_dense(gclib):
    # K_600: colors reach 599, beyond the 512-color window of the work-item path
    ref = assert_parity(gclib, gg.complete(600), 9, check_stats=False)
    assert ref.ncolors == 600 and ref.rounds == 600


@pytest.mark.parametrize("opt", [
    dict(small_max_degree=1), dict(small_max_degree=8), dict(small_max_degree=63), dict(chunk=32),
    dict(chunk=64), dict(chunk=256), dict(chunk=1024), dict(blocks_per_sm=1), dict(blocks_per_sm=2),
    dict(small_max_degree=4, chunk=32, blocks_per_sm=1),
])
def test_launch_configuration_invariance(gclib, opt):
    g = gg.rmat(13, 16, 2)
    assert_parity(gclib, g, 7, options=gclib.Options(**opt))


def test_host_arrays_match_device(gclib):
    g = gg.rmat(12, 16, 2)
    ref = oracle.det(g, 7)
    r = gclib.color(g.rowptr, g.colidx, "det", 7)  # numpy in, numpy out (staged by the library)
    assert isinstance(r.colors, np.ndarray)
    np.testing.assert_array_equal(r.colors, ref.colors)
    assert (r.ncolors, r.rounds) == (ref.ncolors, ref.rounds)


def test_zero_vertices(gclib):
    r = gclib.color(np.zeros(1, np.int32), np.zeros(0, np.int32), "det", 1)
    assert (r.ncolors, r.rounds) == (0, 0)


def test_repeatable_and_properties(gclib):
    g = gg.rmat(14, 16, 2)
    a = run_det(gclib, g, 7)
    b = run_det(gclib, g, 7)
    np.testing.assert_array_equal(a[0], b[0])
    colors = a[0]
    assert oracle.count_conflicts(g, colors) == 0
    assert np.all(colors <= g.degrees())
    assert a[2] >= colors.max() + 1  # a color c first appears in round c+1 or later


@pytest.mark.parametrize("make", [lambda: gg.rmat(14, 16, 2), lambda: gg.complete(600), lambda: gg.star(5000),
                                  lambda: gg.workload("er10k"), lambda: gg.stencil27(9), lambda: gg.crown(40)])
def test_full_sweep_matches_oracle(gclib, make):
    # the full sweep (every entry every round) and the default compact sweep (only neighbours that
    # can still change) are the same method
    g = make()
    ref = oracle.det(g, 11)
    for opt in (gclib.Options(flags=gclib.FLAG_FULL_SWEEP), gclib.Options(flags=gclib.FLAG_FULL_SWEEP, chunk=128),
                gclib.Options(chunk=32, small_max_degree=4), gclib.Options(chunk=1024),
                gclib.Options(chunk=32, small_max_degree=4, core_vertices=-1),
                gclib.Options(chunk=32, small_max_degree=4, core_vertices=max(1, g.n // 20)),
                gclib.Options(chunk=128, core_vertices=max(1, g.n // 5)),
                gclib.Options(chunk=32, small_max_degree=4, core_entries=max(1, g.nnz // 20))):
        c, nc, rounds, st = run_det(gclib, g, 11, options=opt, stats=True)
        np.testing.assert_array_equal(c, ref.colors)
        assert (nc, rounds) == (ref.ncolors, ref.rounds)
        np.testing.assert_array_equal(st.wl_size, ref.wl_size)
        np.testing.assert_array_equal(st.wl_degsum, ref.wl_degsum)


def test_compact_reads_fewer_entries(gclib):
    g = gg.rmat(15, 16, 2)
    _, _, _, full = run_det(gclib, g, 7, options=gclib.Options(flags=gclib.FLAG_FULL_SWEEP), stats=True)
    _, _, _, compact = run_det(gclib, g, 7, stats=True)
    assert full.entries_scanned == full.wl_degsum.sum()
    assert compact.entries_scanned < 0.8 * full.entries_scanned
    # per round: the full sweep reads every entry of the worklist's rows, the compact one a subset
    np.testing.assert_array_equal(full.round_reads, full.wl_degsum)
    assert compact.round_reads.sum() == compact.entries_scanned
    assert (compact.round_reads <= compact.wl_degsum).all()
    # round 1 (every color 0) in the round kernel (this graph would otherwise go to the core phase
    # from round 1): a sweep stops at the first smaller-key neighbour, which for most vertices of a
    # power-law graph comes early in the row
    _, _, _, rk = run_det(gclib, g, 7, options=gclib.Options(core_vertices=-1), stats=True)
    assert rk.round_reads[0] < 0.5 * rk.wl_degsum[0]


def test_batch_full_sweep(gclib):
    import torch
    gs = [gg.rmat(11, 12, 5), gg.complete(300), gg.empty(3), gg.star(2000), gg.workload("er10k")]
    b = gg.pack(gs)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    colors, nc, rd = gclib.color_batch(dev(b.vtx_off), dev(b.edge_off), dev(b.rowptr), dev(b.colidx), "det", 3,
                                       options=gclib.Options(flags=gclib.FLAG_FULL_SWEEP))
    colors = colors.cpu().numpy()
    for i, g in enumerate(gs):
        ref = oracle.det(g, 3)
        np.testing.assert_array_equal(colors[b.vtx_off[i]:b.vtx_off[i + 1]], ref.colors)
        assert (nc[i], rd[i]) == (ref.ncolors, ref.rounds)


# ---------------------------------------------------------------------------------------------
# largest-first priority

LF_GRAPHS = [lambda: gg.star(5000), lambda: gg.crown(40), lambda: gg.grid5(37, 29), lambda: gg.stencil27(9),
             lambda: gg.er(3000, 12.0, 5), lambda: gg.rmat(12, 16, 2), lambda: gg.rmat(15, 16, 2)]


@pytest.mark.parametrize("make", LF_GRAPHS)
@pytest.mark.parametrize("seed", [1, 7])
def test_largest_first_matches_oracle(gclib, make, seed):
    g = make()
    ref = oracle.det(g, seed, priority=oracle.PRIORITY_LARGEST_FIRST)
    assert ref.status == 0
    opt = gclib.Options(priority=gclib.PRIORITY_LARGEST_FIRST)
    colors, nc, rounds, st = run_det(gclib, g, seed, options=opt, stats=True)
    np.testing.assert_array_equal(colors, ref.colors)
    assert (nc, rounds) == (ref.ncolors, ref.rounds)
    np.testing.assert_array_equal(st.wl_size, ref.wl_size)
    np.testing.assert_array_equal(st.wl_degsum, ref.wl_degsum)


def test_largest_first_batch_matches_oracle(gclib):
    import torch
    graphs = [gg.rmat(11, 8, 1), gg.star(300), gg.er(1500, 9.0, 2), gg.grid5(20, 20)]
    b = gg.pack(graphs)
    args = [torch.from_numpy(a).cuda() for a in (b.vtx_off, b.edge_off, b.rowptr, b.colidx)]
    colors, nc, rounds = gclib.color_batch(*args, "det", 7,
                                           options=gclib.Options(priority=gclib.PRIORITY_LARGEST_FIRST))
    colors = colors.cpu().numpy()
    for i, g in enumerate(graphs):
        ref = oracle.det(g, 7, priority=oracle.PRIORITY_LARGEST_FIRST)
        v0, v1 = int(b.vtx_off[i]), int(b.vtx_off[i + 1])
        np.testing.assert_array_equal(colors[v0:v1], ref.colors)
        assert (int(nc[i]), int(rounds[i])) == (ref.ncolors, ref.rounds)


def test_largest_first_inplace_proper(gclib):
    import torch
    g = gg.rmat(15, 16, 3)
    rp, ci = _dev(g)
    r = gclib.color(rp, ci, "inplace", 7, options=gclib.Options(priority=gclib.PRIORITY_LARGEST_FIRST))
    c = r.colors.cpu().numpy()
    assert oracle.count_conflicts(g, c) == 0
    assert np.all(c <= g.degrees()) and r.ncolors == oracle.distinct_colors(c)


def test_unknown_priority_rejected(gclib):
    g = gg.path(10)
    with pytest.raises(gclib.GCError) as e:
        gclib.color(g.rowptr, g.colidx, "det", 1, options=gclib.Options(priority=9))
    assert e.value.status == gclib.GC_ERR_INVALID_ARG


@pytest.mark.parametrize("bps", [3, 4, 2])
@pytest.mark.parametrize("make", [lambda: gg.rmat(14, 16, 2), lambda: gg.stencil27(12)])
def test_kernel_variants_match_oracle(gclib, make, bps):
    # 3: the 80-register variant; 4: the 64-register one; 2: the 64-register one with fewer blocks
    assert_parity(gclib, make(), 7, options=gclib.Options(blocks_per_sm=bps))


# ---------------------------------------------------------------------------------------------
# colors past the 512-color window (the full-row rescan)

def _clique_plus_er(k, n, d, seed):
    """K_k on vertices 0..k-1 plus an Erdos-Renyi part on k..n-1 joined to the clique by random edges."""
    rng = np.random.default_rng(seed)
    edges = [(i, j) for i in range(k) for j in range(i + 1, k)]
    m = int(n * d / 2)
    u = rng.integers(0, n, m)
    v = rng.integers(k, n, m)
    edges += [(int(a), int(b)) for a, b in zip(u, v) if a != b]
    return gg.from_edges(n, edges, name=f"K{k}+ER")


@pytest.mark.parametrize("make", [lambda: gg.complete(600), lambda: gg.complete(1100),
                                  lambda: _clique_plus_er(700, 20000, 12.0, 3)])
@pytest.mark.parametrize("full", [False, True])
def test_colors_beyond_window(gclib, make, full):
    g = make()
    opt = gclib.Options(flags=gclib.FLAG_FULL_SWEEP) if full else None
    ref = assert_parity(gclib, g, 7, options=opt)
    assert ref.ncolors > 512


def test_colors_beyond_window_inplace(gclib):
    g = _clique_plus_er(700, 20000, 12.0, 3)
    rp, ci = _dev(g)
    r = gclib.color(rp, ci, "inplace", 7)
    c = r.colors.cpu().numpy()
    assert oracle.count_conflicts(g, c) == 0
    assert np.all(c <= g.degrees()) and r.ncolors >= 700


# ---------------------------------------------------------------------------------------------
# ordered mode: no speculation, First Fit in key order

ORDERED_GRAPHS = [lambda: gg.complete(40), lambda: gg.complete(600), lambda: gg.star(5000), lambda: gg.crown(40),
                  lambda: gg.empty(33), lambda: gg.grid5(37, 29), lambda: gg.stencil27(9),
                  lambda: gg.er(3000, 12.0, 5), lambda: gg.rmat(12, 16, 2), lambda: gg.rmat(15, 16, 2)]


@pytest.mark.parametrize("make", ORDERED_GRAPHS)
@pytest.mark.parametrize("prio", [0, 1])
def test_ordered_equals_keyorder_greedy(gclib, make, prio):
    g = make()
    colors_ref, k = oracle.greedy_keyorder(g, 7, prio)
    rp, ci = _dev(g)
    depth, deepest = oracle.keyorder_depth(g, 7, prio)
    deg = g.degrees()
    for opt in [dict(priority=prio), dict(priority=prio, flags=gclib.FLAG_FULL_SWEEP),
                dict(priority=prio, small_max_degree=3, chunk=64), dict(priority=prio, blocks_per_sm=1)]:
        r = gclib.color(rp, ci, "ordered", 7, options=gclib.Options(**opt), stats=True)
        np.testing.assert_array_equal(r.colors.cpu().numpy(), colors_ref, err_msg=str(opt))
        assert r.ncolors == oracle.distinct_colors(colors_ref)
        # a vertex is colored in the round after its last smaller-key neighbour
        assert r.rounds == max(deepest, 1)
        if deepest > 0:
            want = [int(np.sum(depth == d)) for d in range(1, deepest + 1)]
            want_deg = [int(deg[depth == d].sum()) for d in range(1, deepest + 1)]
            np.testing.assert_array_equal(r.stats.wl_size, want)
            np.testing.assert_array_equal(r.stats.wl_degsum, want_deg)


def test_ordered_batch_equals_keyorder_greedy(gclib):
    import torch
    graphs = [gg.rmat(11, 8, 1), gg.star(300), gg.empty(5), gg.er(1500, 9.0, 2), gg.complete(70)]
    b = gg.pack(graphs)
    args = [torch.from_numpy(a).cuda() for a in (b.vtx_off, b.edge_off, b.rowptr, b.colidx)]
    colors, nc, rounds = gclib.color_batch(*args, "ordered", 7)
    colors = colors.cpu().numpy()
    for i, g in enumerate(graphs):
        ref, _ = oracle.greedy_keyorder(g, 7)
        v0, v1 = int(b.vtx_off[i]), int(b.vtx_off[i + 1])
        np.testing.assert_array_equal(colors[v0:v1], ref)
        assert int(nc[i]) == oracle.distinct_colors(ref)
        _, deepest = oracle.keyorder_depth(g, 7)
        assert int(rounds[i]) == max(deepest, 1)


# ---------------------------------------------------------------------------------------------
# recoloring pass (iterated greedy over the classes of a given coloring)

RECOLOR_GRAPHS = [lambda: gg.complete(40), lambda: gg.star(5000), lambda: gg.crown(40), lambda: gg.empty(33),
                  lambda: gg.grid5(37, 29), lambda: gg.stencil27(9), lambda: gg.er(3000, 12.0, 5),
                  lambda: gg.rmat(12, 16, 2), lambda: gg.rmat(15, 16, 2)]


@pytest.mark.parametrize("make", RECOLOR_GRAPHS)
def test_recolor_equals_oracle(gclib, make):
    import torch
    g = make()
    rp, ci = _dev(g)
    start = gclib.color(rp, ci, "det", 7)
    cin = start.colors
    ref, k = oracle.greedy_keyorder(g, 3, oracle.PRIORITY_RECOLOR, cin.cpu().numpy())
    _, deepest = oracle.keyorder_depth(g, 3, oracle.PRIORITY_RECOLOR, cin.cpu().numpy())
    for opt in [dict(), dict(small_max_degree=3, chunk=64)]:
        r = gclib.recolor(rp, ci, cin, 3, options=gclib.Options(**opt))
        np.testing.assert_array_equal(r.colors.cpu().numpy(), ref, err_msg=str(opt))
        assert r.ncolors == oracle.distinct_colors(ref) <= start.ncolors
        assert r.rounds == (max(deepest, 1) if g.n else 0)
    # host arrays in and out, and the input array reused as the output
    rh = gclib.recolor(g.rowptr, g.colidx, cin.cpu().numpy(), 3)
    np.testing.assert_array_equal(rh.colors, ref)
    same = cin.clone()
    gclib.recolor(rp, ci, same, 3, out=same)
    np.testing.assert_array_equal(same.cpu().numpy(), ref)


def test_recolor_passes_never_add_colors(gclib):
    g = gg.rmat(15, 16, 2)
    rp, ci = _dev(g)
    r = gclib.color(rp, ci, "inplace", 7)
    counts = [r.ncolors]
    c = r.colors
    for it in range(5):
        ref, _ = oracle.greedy_keyorder(g, it, oracle.PRIORITY_RECOLOR, c.cpu().numpy())
        r = gclib.recolor(rp, ci, c, it)
        np.testing.assert_array_equal(r.colors.cpu().numpy(), ref)
        counts.append(r.ncolors)
        c = r.colors
    assert counts == sorted(counts, reverse=True) and counts[-1] < counts[0]


def test_recolor_rejects_negative_colors(gclib):
    import torch
    g = gg.er(500, 6.0, 1)
    rp, ci = _dev(g)
    cin = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    cin[123] = -1
    with pytest.raises(gclib.GCError) as e:
        gclib.recolor(rp, ci, cin, 1)
    assert e.value.status == gclib.GC_ERR_INVALID_ARG


# ---------------------------------------------------------------------------------------------
# smallest-last order (batch peeling) and colorings under its key

SL_GRAPHS = [lambda: gg.path(2), lambda: gg.path(97), lambda: gg.star(5000), lambda: gg.cycle(1000),
             lambda: gg.complete(40), lambda: gg.complete(600), lambda: gg.empty(33), lambda: gg.crown(40),
             lambda: gg.grid5(37, 29), lambda: gg.stencil27(9), lambda: gg.er(3000, 12.0, 5),
             lambda: gg.rmat(12, 16, 2), lambda: gg.rmat(15, 16, 2)]


@pytest.mark.parametrize("make", SL_GRAPHS)
def test_smallest_last_levels_equal_oracle(gclib, make):
    g = make()
    ref, k = oracle.peel_levels(g)
    rp, ci = _dev(g)
    for opt in [dict(), dict(small_max_degree=3, chunk=64)]:
        level, nlevels, degen = gclib.smallest_last(rp, ci, options=gclib.Options(**opt))
        np.testing.assert_array_equal(level.cpu().numpy(), ref, err_msg=str(opt))
        assert nlevels == (int(ref.max()) if g.n else 0) and degen == k
    level_h, _, _ = gclib.smallest_last(g.rowptr, g.colidx)  # host arrays
    np.testing.assert_array_equal(level_h, ref)


@pytest.mark.parametrize("make", SL_GRAPHS[-6:])
def test_smallest_last_colorings_equal_oracle(gclib, make):
    g = make()
    rp, ci = _dev(g)
    sl = gclib.Options(priority=gclib.PRIORITY_SMALLEST_LAST)
    # deterministic speculative mode: bit-exact, with the per-round worklists
    ref = oracle.det(g, 7, priority=oracle.PRIORITY_SMALLEST_LAST)
    r = gclib.color(rp, ci, "det", 7, options=sl, stats=True)
    np.testing.assert_array_equal(r.colors.cpu().numpy(), ref.colors)
    assert (r.ncolors, r.rounds) == (ref.ncolors, ref.rounds)
    np.testing.assert_array_equal(r.stats.wl_size, ref.wl_size)
    # ordered mode: First Fit in smallest-last order, at most degeneracy + 1 colors
    _, k = oracle.peel_levels(g)
    cref, nc = oracle.greedy_keyorder(g, 7, oracle.PRIORITY_SMALLEST_LAST)
    _, deepest = oracle.keyorder_depth(g, 7, oracle.PRIORITY_SMALLEST_LAST)
    r = gclib.color(rp, ci, "ordered", 7, options=sl)
    np.testing.assert_array_equal(r.colors.cpu().numpy(), cref)
    assert r.ncolors == nc <= k + 1 and r.rounds == max(deepest, 1)
    # in-place mode: the invariants
    r = gclib.color(rp, ci, "inplace", 7, options=sl)
    c = r.colors.cpu().numpy()
    assert oracle.count_conflicts(g, c) == 0 and np.all(c <= g.degrees())


def test_smallest_last_rejects_batches_and_bad_graphs(gclib):
    import torch
    graphs = [gg.er(300, 5.0, 1), gg.star(20)]
    b = gg.pack(graphs)
    args = [torch.from_numpy(a).cuda() for a in (b.vtx_off, b.edge_off, b.rowptr, b.colidx)]
    with pytest.raises(gclib.GCError) as e:
        gclib.color_batch(*args, "det", 7, options=gclib.Options(priority=gclib.PRIORITY_SMALLEST_LAST))
    assert e.value.status == gclib.GC_ERR_INVALID_ARG
    g = gg.from_edges(5, [(0, 1), (1, 2)])
    ci = g.colidx.copy()
    ci[0] = 0  # a self-loop at vertex 0
    with pytest.raises(gclib.GCError) as e:
        gclib.smallest_last(g.rowptr, ci)
    assert e.value.status == gclib.GC_ERR_INVALID_GRAPH
