"""In-place mode invariants, batched coloring and boundary errors on the GPU.

In-place mode reads neighbour colors live (as the paper's threads do, Algorithm 1 phase 1), so its
coloring is not unique: it is checked for what Lemma 1 and Section 2.1 fix (a proper coloring,
color(v) <= deg(v), hence at most Delta+1 colors) and for termination within n rounds.  Batched
deterministic coloring must equal the oracle per graph, bit for bit."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_inplace(gc, g, seed=3):
    r = gc.color(_dev(g.rowptr), _dev(g.colidx if g.nnz else np.zeros(0, np.int32)), "inplace", seed)
    c = r.colors.cpu().numpy()
    assert oracle.count_conflicts(g, c) == 0, g.name
    if g.n:
        assert c.min() >= 0
        assert np.all(c <= g.degrees())
    assert r.ncolors == oracle.distinct_colors(c)
    assert (g.n == 0 and r.rounds == 0) or 1 <= r.rounds <= g.n
    return r


@pytest.mark.parametrize("make", [
    lambda: gg.complete(70), lambda: gg.complete(600), lambda: gg.star(3000), lambda: gg.cycle(1001),
    lambda: gg.crown(50), lambda: gg.empty(10), lambda: gg.stencil27(12), lambda: gg.workload("er10k"),
    lambda: gg.rmat(15, 16, 2), lambda: gg.grid5(100, 37),
])
def test_inplace_invariants(gclib, make):
    check_inplace(gclib, make())


def test_inplace_options(gclib):
    # the compact sweep (default) with many items per vertex, many larger vertices and list rewrites;
    # the full sweep; both kernel variants
    g = gg.rmat(13, 16, 2)
    for opt in [dict(small_max_degree=2), dict(chunk=32), dict(blocks_per_sm=1), dict(blocks_per_sm=3),
                dict(blocks_per_sm=4), dict(flags=gclib.FLAG_FULL_SWEEP), dict(small_max_degree=1, chunk=64),
                dict(flags=gclib.FLAG_FULL_SWEEP, chunk=32)]:
        r = gclib.color(_dev(g.rowptr), _dev(g.colidx), "inplace", 1, options=gclib.Options(**opt))
        c = r.colors.cpu().numpy()
        assert oracle.count_conflicts(g, c) == 0, opt
        assert np.all(c <= g.degrees()) and r.ncolors == oracle.distinct_colors(c), opt


@pytest.mark.parametrize("make", [lambda: gg.rmat(16, 16, 4), lambda: gg.complete(1100), lambda: gg.star(70000)])
def test_inplace_compact_stress(gclib, make):
    # larger vertices with long lists: rewrites, several items per vertex, colors past 512
    g = make()
    for opt in [dict(), dict(small_max_degree=3, chunk=64)]:
        r = gclib.color(_dev(g.rowptr), _dev(g.colidx), "inplace", 5, options=gclib.Options(**opt))
        c = r.colors.cpu().numpy()
        assert oracle.count_conflicts(g, c) == 0, opt
        assert np.all(c <= g.degrees()) and r.ncolors == oracle.distinct_colors(c)
        assert 1 <= r.rounds <= g.n


def _mixed_graphs():
    gs = [gg.complete(3), gg.empty(4), gg.star(40), gg.workload("er10k"), gg.rmat(12, 12, 5), gg.cycle(9),
          gg.crown(20), gg.complete(300), gg.stencil27(5), gg.empty(1), gg.path(2)]
    gs += [gg.make_from_spec(s) for s in gg.batch_specs(12, 3, nmin=100, nmax=20_000)]
    return gs


def test_batch_det_matches_oracle_per_graph(gclib):
    gs = _mixed_graphs()
    b = gg.pack(gs)
    colors, nc, rd = gclib.color_batch(_dev(b.vtx_off), _dev(b.edge_off), _dev(b.rowptr), _dev(b.colidx), "det", 7)
    colors = colors.cpu().numpy()
    for i, g in enumerate(gs):
        ref = oracle.det(g, 7)
        np.testing.assert_array_equal(colors[b.vtx_off[i]:b.vtx_off[i + 1]], ref.colors, err_msg=f"graph {i}")
        assert nc[i] == ref.ncolors and rd[i] == ref.rounds, (i, nc[i], ref.ncolors, rd[i], ref.rounds)


@pytest.mark.parametrize("opt", [dict(tail_vertices=-1), dict(tail_vertices=4096), dict(core_vertices=-1),
                                 dict(core_vertices=3000, tail_vertices=200)])
def test_batch_det_phases_match_oracle(gclib, opt):
    # the batch through the round kernel, the core phase and the tail phase, with the hand-overs at
    # other points than the default's
    gs = _mixed_graphs()
    b = gg.pack(gs)
    colors, nc, rd = gclib.color_batch(_dev(b.vtx_off), _dev(b.edge_off), _dev(b.rowptr), _dev(b.colidx), "det", 7,
                                       options=gclib.Options(**opt))
    colors = colors.cpu().numpy()
    for i, g in enumerate(gs):
        ref = oracle.det(g, 7)
        np.testing.assert_array_equal(colors[b.vtx_off[i]:b.vtx_off[i + 1]], ref.colors, err_msg=f"{opt} graph {i}")
        assert nc[i] == ref.ncolors and rd[i] == ref.rounds, (opt, i)


def test_batch_round_statistics_are_sums_over_graphs(gclib):
    # the batch's worklist in round r is the union of the graphs' worklists in round r
    gs = _mixed_graphs()
    b = gg.pack(gs)
    _, _, rd, st = gclib.color_batch(_dev(b.vtx_off), _dev(b.edge_off), _dev(b.rowptr), _dev(b.colidx), "det", 7,
                                     stats=True)
    R = int(max(rd))
    want_w = np.zeros(R, np.int64)
    want_d = np.zeros(R, np.int64)
    for g in gs:
        ref = oracle.det(g, 7)
        want_w[:len(ref.wl_size)] += ref.wl_size
        want_d[:len(ref.wl_degsum)] += ref.wl_degsum
    assert st.rounds == R
    np.testing.assert_array_equal(st.wl_size, want_w)
    np.testing.assert_array_equal(st.wl_degsum, want_d)


def test_batch_host_arrays_and_empty_graphs(gclib):
    gs = [gg.empty(0), gg.complete(4), gg.empty(0), gg.cycle(5), gg.empty(0)]
    b = gg.pack(gs)
    colors, nc, rd = gclib.color_batch(b.vtx_off, b.edge_off, b.rowptr, b.colidx, "det", 1)
    assert list(nc) == [0, 4, 0, 3, 0]
    assert rd[0] == 0 and rd[2] == 0 and rd[4] == 0
    for i, g in enumerate(gs):
        ref = oracle.det(g, 1)
        np.testing.assert_array_equal(colors[b.vtx_off[i]:b.vtx_off[i + 1]], ref.colors)
        assert rd[i] == ref.rounds


def test_batch_inplace_proper(gclib):
    gs = _mixed_graphs()
    b = gg.pack(gs)
    colors, nc, rd = gclib.color_batch(_dev(b.vtx_off), _dev(b.edge_off), _dev(b.rowptr), _dev(b.colidx),
                                       "inplace", 7)
    colors = colors.cpu().numpy()
    for i, g in enumerate(gs):
        c = colors[b.vtx_off[i]:b.vtx_off[i + 1]]
        assert oracle.count_conflicts(g, c) == 0
        assert nc[i] == oracle.distinct_colors(c)


def test_batch_equals_solo(gclib):
    gs = [gg.make_from_spec(s) for s in gg.batch_specs(8, 3, nmin=1000, nmax=50_000)]
    b = gg.pack(gs)
    colors, nc, rd = gclib.color_batch(_dev(b.vtx_off), _dev(b.edge_off), _dev(b.rowptr), _dev(b.colidx), "det", 7)
    colors = colors.cpu().numpy()
    for i, g in enumerate(gs):
        r = gclib.color(_dev(g.rowptr), _dev(g.colidx), "det", 7)
        np.testing.assert_array_equal(colors[b.vtx_off[i]:b.vtx_off[i + 1]], r.colors.cpu().numpy())
        assert (nc[i], rd[i]) == (r.ncolors, r.rounds)


# ---------------------------------------------------------------------------------------------
# boundary errors: right status, outputs untouched, device still usable

def _expect(gc, status, rowptr, colidx, mode="det", **kw):
    out = np.full(max(len(rowptr) - 1, 1), -77, np.int32)[: max(len(rowptr) - 1, 0)]
    with pytest.raises(gc.GCError) as ei:
        gc.color(rowptr, colidx, mode, 1, out=out, **kw)
    assert ei.value.status == status, str(ei.value)
    assert np.all(out == -77)


@pytest.mark.parametrize("mode", ["det", "inplace"])
def test_malformed_graphs(gclib, mode):
    ok = gg.cycle(6)
    bad = ok.colidx.copy()
    bad[3] = 6  # out of range
    _expect(gclib, gclib.GC_ERR_INVALID_GRAPH, ok.rowptr, bad, mode)
    bad = ok.colidx.copy()
    bad[0] = -1
    _expect(gclib, gclib.GC_ERR_INVALID_GRAPH, ok.rowptr, bad, mode)
    bad = ok.colidx.copy()
    bad[0] = 0  # self-loop on vertex 0
    _expect(gclib, gclib.GC_ERR_INVALID_GRAPH, ok.rowptr, bad, mode)
    rp = ok.rowptr.copy()
    rp[2], rp[3] = rp[3], rp[2]  # non-monotone
    _expect(gclib, gclib.GC_ERR_INVALID_GRAPH, rp, ok.colidx, mode)
    rp = ok.rowptr.copy()
    rp[0] = 1
    _expect(gclib, gclib.GC_ERR_INVALID_GRAPH, rp, ok.colidx, mode)
    # big graph with one bad entry deep inside a hub row (work-item path)
    g = gg.star(4000)
    bad = g.colidx.copy()
    bad[3000] = 0
    _expect(gclib, gclib.GC_ERR_INVALID_GRAPH, g.rowptr, bad, mode)
    # the device is still usable
    r = gclib.color(ok.rowptr, ok.colidx, mode, 1)
    assert r.ncolors == 2


def test_bad_arguments(gclib):
    with pytest.raises(gclib.GCError) as ei:
        gclib.color(np.zeros(3, np.int32), np.zeros(0, np.int32), "det", 1, options=gclib.Options(chunk=48))
    assert ei.value.status == gclib.GC_ERR_INVALID_ARG
    with pytest.raises(gclib.GCError) as ei:
        gclib.color(np.zeros(3, np.int32), np.zeros(0, np.int32), 5, 1)
    assert ei.value.status == gclib.GC_ERR_INVALID_ARG
    lib = gclib.load()
    assert lib.gc_color(-1, None, None, 0, 0, None, None, None) == gclib.GC_ERR_INVALID_ARG
    assert lib.gc_color(3, None, None, 0, 0, None, None, None) == gclib.GC_ERR_INVALID_ARG


@pytest.mark.parametrize("mode", ["det", "inplace"])
def test_round_cap(gclib, mode):
    g = gg.complete(10)  # needs 10 rounds in deterministic mode
    if mode == "det":
        _expect(gclib, gclib.GC_ERR_NO_CONVERGENCE, g.rowptr, g.colidx, mode, options=gclib.Options(max_rounds=3))
    r = gclib.color(g.rowptr, g.colidx, mode, 1, options=gclib.Options(max_rounds=10))
    assert r.ncolors == 10


@pytest.mark.parametrize("mode", ["det", "inplace", "ordered", "partition"])
def test_barrier_wait_limit(gclib, mode):
    # a 1 ns limit makes every early block give up at the first grid barrier: the call must
    # report GC_ERR_TIMEOUT, leave the output untouched, and the next call must work
    g = gg.rmat(14, 16, 2)
    _expect(gclib, gclib.GC_ERR_TIMEOUT, g.rowptr, g.colidx, mode, options=gclib.Options(spin_limit_ns=1))
    ref = oracle.det(g, 1)
    r = gclib.color(g.rowptr, g.colidx, "det", 1)
    np.testing.assert_array_equal(r.colors, ref.colors)


def test_validate(gclib):
    g = gg.rmat(10, 8, 1)
    gclib.validate(g.rowptr, g.colidx)
    # asymmetric: drop one direction of an edge
    v = 5
    row = g.colidx[g.rowptr[v]:g.rowptr[v + 1]]
    u = int(row[0])
    keep = np.ones(g.nnz, bool)
    keep[g.rowptr[v]] = False
    rp = g.rowptr.copy()
    rp[v + 1:] -= 1
    with pytest.raises(gclib.GCError) as ei:
        gclib.validate(rp, g.colidx[keep])
    assert ei.value.status == gclib.GC_ERR_INVALID_GRAPH
    assert u >= 0
    # unsorted row
    ci = g.colidx.copy()
    big = int(np.argmax(g.degrees()))
    a, b = g.rowptr[big], g.rowptr[big + 1]
    ci[a:b] = ci[a:b][::-1]
    with pytest.raises(gclib.GCError):
        gclib.validate(g.rowptr, ci, gclib.VALIDATE_SORTED)
    gclib.validate(g.rowptr, ci, 0)  # range and self-loop checks alone pass


def test_smallest_last_barrier_wait_limit(gclib):
    # the peeling kernel's grid barriers give up the same way; the next call works
    g = gg.rmat(14, 16, 2)
    with pytest.raises(gclib.GCError) as ei:
        gclib.smallest_last(g.rowptr, g.colidx, options=gclib.Options(spin_limit_ns=1))
    assert ei.value.status == gclib.GC_ERR_TIMEOUT
    level, _, k = gclib.smallest_last(g.rowptr, g.colidx)
    ref, kref = oracle.peel_levels(g)
    np.testing.assert_array_equal(level, ref)
    assert k == kref


def test_ordered_round_cap_and_bad_input(gclib):
    g = gg.complete(10)  # the keys form one chain: 10 rounds
    _expect(gclib, gclib.GC_ERR_NO_CONVERGENCE, g.rowptr, g.colidx, "ordered", options=gclib.Options(max_rounds=3))
    assert gclib.color(g.rowptr, g.colidx, "ordered", 1, options=gclib.Options(max_rounds=10)).ncolors == 10
    ok = gg.cycle(6)
    bad = ok.colidx.copy()
    bad[3] = 6  # out of range
    _expect(gclib, gclib.GC_ERR_INVALID_GRAPH, ok.rowptr, bad, "ordered")
    # asymmetric: vertex 1 lists 0 but 0 lists nothing; with key(0) < key(1), vertex 1 waits for a
    # release that never comes, which the kernel reports once the ready lists run dry
    seed = next(s for s in range(100) if oracle.key_less(s, 0, 1))
    rp = np.array([0, 0, 1], np.int32)
    ci = np.array([0], np.int32)
    out = np.full(2, -77, np.int32)
    with pytest.raises(gclib.GCError) as ei:
        gclib.color(rp, ci, "ordered", seed, out=out)
    assert ei.value.status == gclib.GC_ERR_INVALID_GRAPH and np.all(out == -77)


@pytest.mark.parametrize("mode,prio", [("det", 0), ("det", 2), ("inplace", 0), ("ordered", 0), ("ordered", 2),
                                       ("partition", 0)])
def test_host_arrays_every_mode(gclib, mode, prio):
    # host CSR arrays are uploaded beside the set-up kernels; every path must wait for the upload
    # before its first kernel that reads the adjacency (deterministic paths: identical colors)
    import torch
    g = gg.rmat(14, 16, 3)
    opt = gclib.Options(priority=prio)
    rh = gclib.color(g.rowptr, g.colidx, mode, 5, options=opt)
    rd = gclib.color(torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.colidx).cuda(), mode, 5, options=opt)
    assert isinstance(rh.colors, np.ndarray)
    if mode == "inplace":
        assert oracle.count_conflicts(g, rh.colors) == 0 and np.all(rh.colors <= g.degrees())
    else:
        np.testing.assert_array_equal(rh.colors, rd.colors.cpu().numpy())
        assert (rh.ncolors, rh.rounds) == (rd.ncolors, rd.rounds)
