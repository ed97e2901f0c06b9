"""Full-size workloads in the launch configuration bench.py times (library defaults).

Deterministic mode: the whole coloring of R-MAT scale 22 and of the 256^3 27-point stencil is
compared with the CPU oracle entry by entry (the oracle takes about a minute for each).  In-place
mode: the invariants that hold at any size (Lemma 1: proper; Section 2.1: color(v) <= deg(v), so at
most Delta+1 colors; at most n rounds)."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SEED = 7  # the benchmark's hash seed


@pytest.fixture(scope="module", params=["rmat22", "stencil256"])
def full(request):
    import torch
    g = gg.workload(request.param)
    return g, torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.colidx).cuda()


@pytest.fixture(scope="module")
def full_ref(full):
    g, _, _ = full
    ref = oracle.det(g, SEED)
    assert ref.status == 0
    return ref


@pytest.mark.parametrize("core", [0, -1, 20_000], ids=["core-default", "core-off", "core-20k"])
def test_full_size_deterministic_matches_oracle(gclib, full, full_ref, core):
    # the library default hands the last rounds to the shared-memory core phase; -1 keeps every
    # round in the regular round kernel; 20k hands over later
    g, rp, ci = full
    ref = full_ref
    r = gclib.color(rp, ci, "det", SEED, stats=True, round_cap=1 << 12, options=gclib.Options(core_vertices=core))
    np.testing.assert_array_equal(r.colors.cpu().numpy(), ref.colors)
    assert (r.ncolors, r.rounds) == (ref.ncolors, ref.rounds)
    np.testing.assert_array_equal(r.stats.wl_size, ref.wl_size)
    np.testing.assert_array_equal(r.stats.wl_degsum, ref.wl_degsum)


def test_full_size_inplace_invariants(gclib, full):
    g, rp, ci = full
    r = gclib.color(rp, ci, "inplace", SEED)
    c = r.colors.cpu().numpy()
    assert oracle.count_conflicts(g, c) == 0
    assert c.min() >= 0 and np.all(c <= g.degrees())
    assert r.ncolors == oracle.distinct_colors(c) <= g.max_degree + 1
    assert 1 <= r.rounds <= g.n


def test_full_size_smallest_last_matches_oracle(gclib, full):
    g, rp, ci = full
    level, nlevels, degen = gclib.smallest_last(rp, ci)
    ref, k = oracle.peel_levels(g)
    np.testing.assert_array_equal(level.cpu().numpy(), ref)
    assert (nlevels, degen) == (int(ref.max()), k)
    r = gclib.color(rp, ci, "ordered", SEED, options=gclib.Options(priority=gclib.PRIORITY_SMALLEST_LAST))
    cref, nc = oracle.greedy_keyorder(g, SEED, oracle.PRIORITY_SMALLEST_LAST)
    np.testing.assert_array_equal(r.colors.cpu().numpy(), cref)
    assert r.ncolors == nc <= k + 1
