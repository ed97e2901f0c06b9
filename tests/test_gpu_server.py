"""Continuous-batching server: every request's result equals the oracle (deterministic mode) or is
a proper coloring (in-place mode), whether it ran alone or joined a batch already on the GPU."""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _graphs():
    gs = [gg.complete(7), gg.empty(5), gg.star(300), gg.cycle(11), gg.crown(25), gg.complete(260),
          gg.grid5(30, 20), gg.workload("er10k")]
    gs += [gg.make_from_spec(s) for s in gg.batch_specs(14, 4, nmin=1000, nmax=60_000)]
    return gs


def test_server_det_matches_oracle_staggered(gclib):
    gs = _graphs()
    refs = [oracle.det(g, 7) for g in gs]
    with gclib.Server(pool_vertices=2_000_000, pool_entries=40_000_000, mode="det", seed=7) as srv:
        ids = []
        for i, g in enumerate(gs):
            ids.append(srv.submit(g.rowptr, g.colidx))
            if i % 5 == 4:
                time.sleep(0.002)  # later requests arrive while earlier ones are resident
        for g, ref, rid in zip(gs, refs, ids):
            colors, nc, rounds = srv.poll(rid, timeout_ms=-1)
            np.testing.assert_array_equal(colors, ref.colors, err_msg=g.name)
            assert (nc, rounds) == (ref.ncolors, ref.rounds), g.name
        st = srv.stats()
        assert st["completed"] == len(gs) and st["queued"] == 0 and st["resident"] == 0
        assert st["p99_ms"] >= st["p50_ms"] > 0
        # the batch overlapped requests: fewer batched rounds than rounds summed over requests
        assert st["rounds_run"] < sum(r.rounds for r in refs)


def test_server_small_pool_queues_and_admits(gclib):
    gs = [gg.make_from_spec(s) for s in gg.batch_specs(10, 8, nmin=5000, nmax=30_000)]
    pv = max(g.n for g in gs) + 10
    pe = max(g.nnz for g in gs) + 10
    with gclib.Server(pool_vertices=pv, pool_entries=pe, mode="det", seed=3) as srv:
        ids = [srv.submit(g.rowptr, g.colidx) for g in gs]
        for g, rid in zip(gs, ids):
            colors, nc, rounds = srv.poll(rid)
            ref = oracle.det(g, 3)
            np.testing.assert_array_equal(colors, ref.colors)
            assert rounds == ref.rounds


def test_server_inplace_proper(gclib):
    gs = _graphs()[:12]
    with gclib.Server(pool_vertices=1_000_000, pool_entries=20_000_000, mode="inplace", seed=1) as srv:
        ids = [srv.submit(g.rowptr, g.colidx) for g in gs]
        for g, rid in zip(gs, ids):
            colors, nc, rounds = srv.poll(rid)
            assert oracle.count_conflicts(g, colors) == 0
            assert nc == oracle.distinct_colors(colors)


def test_server_rejects(gclib):
    with gclib.Server(pool_vertices=1000, pool_entries=10_000, mode="det") as srv:
        big = gg.er(5000, 4, 1)
        with pytest.raises(gclib.GCError) as ei:
            srv.submit(big.rowptr, big.colidx)
        assert ei.value.status == gclib.GC_ERR_OOM
        g = gg.cycle(6)
        rp = g.rowptr.copy()
        rp[3] = rp[4] + 1  # row offsets not monotone: refused at submit
        with pytest.raises(gclib.GCError) as ei:
            srv.submit(rp, g.colidx)
        assert ei.value.status == gclib.GC_ERR_INVALID_GRAPH
        bad = g.colidx.copy()
        bad[0] = 0  # self-loop: found on the device at admission, reported by poll
        rid_bad = srv.submit(g.rowptr, bad)
        rid = srv.submit(g.rowptr, g.colidx)
        with pytest.raises(gclib.GCError) as ei:
            srv.poll(rid_bad)
        assert ei.value.status == gclib.GC_ERR_INVALID_GRAPH
        colors, nc, rounds = srv.poll(rid)
        assert nc == 2 and srv.stats()["rejected"] == 2


def test_server_device_inputs(gclib):
    import torch
    g = gg.rmat(12, 16, 2)
    with gclib.Server(pool_vertices=100_000, pool_entries=2_000_000, mode="det", seed=7) as srv:
        rid = srv.submit(torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.colidx).cuda())
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        _, nc, rounds = srv.poll(rid, out=out)
        ref = oracle.det(g, 7)
        np.testing.assert_array_equal(out.cpu().numpy(), ref.colors)


def test_server_mixed_modes_and_seeds(gclib):
    # one server, requests with their own mode and seed (the problem of Section 2.1 with the
    # conflict rule of Algorithm 1 under each request's priority): every deterministic result equals
    # the oracle for its own seed; the in-place one is a proper coloring within Delta + 1 colors
    gs = [gg.rmat(12, 16, 2), gg.workload("er10k"), gg.rmat(11, 12, 5), gg.complete(90), gg.crown(30)]
    seeds = [1, 7, 2**63 + 5, 3, 11]
    with gclib.Server(pool_vertices=500_000, pool_entries=10_000_000, mode="det", seed=0) as srv:
        ids = [srv.submit(g.rowptr, g.colidx, mode="det", seed=sd) for g, sd in zip(gs, seeds)]
        ip_graph = gg.rmat(12, 16, 9)
        ip_id = srv.submit(ip_graph.rowptr, ip_graph.colidx, mode="inplace", seed=5)
        # the same graph under two seeds in the same batch
        twin = srv.submit(gs[0].rowptr, gs[0].colidx, mode="det", seed=99)
        for g, sd, rid in zip(gs, seeds, ids):
            ref = oracle.det(g, sd)
            colors, nc, rounds = srv.poll(rid, timeout_ms=-1)
            np.testing.assert_array_equal(colors, ref.colors, err_msg=f"{g.name} seed {sd}")
            assert (nc, rounds) == (ref.ncolors, ref.rounds)
        ref = oracle.det(gs[0], 99)
        colors, nc, rounds = srv.poll(twin, timeout_ms=-1)
        np.testing.assert_array_equal(colors, ref.colors)
        assert (nc, rounds) == (ref.ncolors, ref.rounds)
        colors, nc, rounds = srv.poll(ip_id, timeout_ms=-1)
        assert oracle.count_conflicts(ip_graph, colors) == 0
        assert np.all(colors <= ip_graph.degrees()) and nc == oracle.distinct_colors(colors)
        st = srv.stats()
        assert st["completed"] == len(gs) + 2 and st["failed"] == 0


def test_server_rejects_unknown_request_mode(gclib):
    g = gg.cycle(9)
    with gclib.Server(pool_vertices=1000, pool_entries=10_000, mode="det") as srv:
        for mode in ("partition", "ordered", 7):
            with pytest.raises(gclib.GCError) as ei:
                srv.submit(g.rowptr, g.colidx, mode=mode)
            assert ei.value.status == gclib.GC_ERR_INVALID_ARG


def test_server_survives_device_error(gclib):
    # every launch's grid-barrier wait runs out (a 1 ns limit): the resident requests end with
    # GC_ERR_TIMEOUT, the pool is reset, and the worker goes on to the next request
    g = gg.rmat(12, 16, 2)
    with gclib.Server(pool_vertices=100_000, pool_entries=2_000_000, mode="det", seed=7, spin_limit_ns=1) as srv:
        for _ in range(2):
            rid = srv.submit(g.rowptr, g.colidx)
            with pytest.raises(gclib.GCError) as ei:
                srv.poll(rid, timeout_ms=-1)
            assert ei.value.status == gclib.GC_ERR_TIMEOUT
        st = srv.stats()
        assert st["failed"] == 2 and st["resident"] == 0 and st["queued"] == 0
    # the device is still usable afterwards
    ref = oracle.det(g, 7)
    r = gclib.color(g.rowptr, g.colidx, "det", 7)
    np.testing.assert_array_equal(r.colors, ref.colors)


def test_server_colors_large_requests_alone(gclib):
    # requests with at least solo_entries adjacency entries skip the pool and are colored alone
    # between batch launches (core and tail phases included); the others keep joining the batch;
    # every result is the one the request would get by itself
    gs = _graphs()
    assert any(g.nnz >= 20_000 for g in gs) and any(g.nnz < 20_000 for g in gs)
    refs = [oracle.det(g, 3) for g in gs]
    big = gg.workload("er10k")
    bad = gg.er(3000, 12.0, 4)
    bad_ci = bad.colidx.copy()
    bad_ci[7] = bad.n + 5  # neighbour id out of range: found by the solo coloring, reported by poll
    with gclib.Server(pool_vertices=2_000_000, pool_entries=40_000_000, mode="det", seed=3,
                      solo_entries=20_000) as srv:
        ids = [srv.submit(g.rowptr, g.colidx) for g in gs]
        rin = srv.submit(big.rowptr, big.colidx, mode="inplace", seed=5)
        rbad = srv.submit(bad.rowptr, bad_ci)
        for g, ref, rid in zip(gs, refs, ids):
            colors, nc, rounds = srv.poll(rid, timeout_ms=-1)
            np.testing.assert_array_equal(colors, ref.colors, err_msg=g.name)
            assert (nc, rounds) == (ref.ncolors, ref.rounds), g.name
        c, nc, _ = srv.poll(rin, timeout_ms=-1)
        assert oracle.count_conflicts(big, c) == 0 and nc == oracle.distinct_colors(c)
        with pytest.raises(gclib.GCError) as ei:
            srv.poll(rbad, timeout_ms=-1)
        assert ei.value.status == gclib.GC_ERR_INVALID_GRAPH
        st = srv.stats()
        assert st["completed"] == len(gs) + 1 and st["rejected"] == 1 and st["queued"] == 0
