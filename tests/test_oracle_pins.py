"""Pins of the CPU oracle to facts fixed outside it (no GPU).

The paper (arXiv:1509.08267) gives definitions and two lemmas but no worked example, so the oracle
is pinned to: published SplitMix64 outputs (the priority hash); closed forms derived by hand from
First Fit (Section 3) and Algorithm 1 (Section 3.1) on complete graphs, stars, complete bipartite
graphs, single edges, cycles, grids, the 27-point stencil and crown graphs; the characterisation
of First Fit; proper coloring (Lemma 1) and the Delta+1 bound (Section 2.1); termination and the
round bound (Lemma 2 and its corollary); and brute-force chromatic numbers on tiny graphs.
"""
import itertools
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------------
# priority hash

def test_splitmix64_published_outputs():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l[0] != "#"]
    for idx, hexval in rows:
        assert oracle.splitmix64(0, int(idx)) == int(hexval, 16)


def test_splitmix64_is_the_stream():
    # output i of the stream seeded s equals output 0 of the stream seeded s + i*GAMMA
    gamma = 0x9E3779B97F4A7C15
    for s in (0, 1, 7, 2**64 - 1):
        for i in (0, 1, 5, 1000):
            assert oracle.splitmix64(s, i) == oracle.splitmix64((s + i * gamma) % 2**64, 0)


def test_key_order_is_total_and_matches_hash_then_id():
    seed = 7
    h = oracle.keys(seed, 64)
    for u in range(64):
        for v in range(64):
            expect = (int(h[u]), u) < (int(h[v]), v)
            assert oracle.key_less(seed, u, v) == expect


# ---------------------------------------------------------------------------------------------
# greedy First Fit (natural order)

def test_greedy_complete():
    for n in (1, 2, 7, 30):
        c, k = oracle.greedy(gg.complete(n))
        assert k == n
        assert list(c) == list(range(n))


def test_greedy_cycles_and_paths():
    for n in (3, 5, 9, 101):
        assert oracle.greedy(gg.cycle(n))[1] == 3  # odd cycle: 0,1,0,1,...,2
    for n in (4, 6, 100):
        c, k = oracle.greedy(gg.cycle(n))
        assert k == 2 and list(c) == [i & 1 for i in range(n)]
    c, k = oracle.greedy(gg.path(10))
    assert list(c) == [i & 1 for i in range(10)]


def test_greedy_grid_checkerboard():
    Lx, Ly = 13, 7
    c, k = oracle.greedy(gg.grid5(Lx, Ly))
    assert k == 2
    x, y = np.meshgrid(np.arange(Lx), np.arange(Ly))
    assert np.array_equal(c, ((x + y) & 1).ravel())


@pytest.mark.parametrize("L", [2, 3, 4, 5])
def test_greedy_stencil27_eight_colors(L):
    # any 2x2x2 block is K_8, so 8 colors are necessary; natural-order First Fit reaches exactly
    # color (x&1) + 2(y&1) + 4(z&1)
    g = gg.stencil27(L)
    c, k = oracle.greedy(g)
    assert k == min(8, 2 ** sum(1 for _ in range(3) if L > 1))
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    assert np.array_equal(c, ((x & 1) + 2 * (y & 1) + 4 * (z & 1)).ravel())


def test_greedy_crown_graph():
    # the textbook worst case: interleaved order forces k colors on a bipartite graph
    for k in (3, 6, 11):
        assert oracle.greedy(gg.crown(k, interleaved=True))[1] == k
        assert oracle.greedy(gg.crown(k, interleaved=False))[1] == 2


def _first_fit_characterisation(g, c):
    """Proper, and every vertex of color k has earlier neighbours of every color < k: this
    determines natural-order First Fit uniquely (induction on the vertex order)."""
    for v in range(g.n):
        nb = g.colidx[g.rowptr[v]:g.rowptr[v + 1]]
        earlier = {int(c[u]) for u in nb if u < v}
        assert int(c[v]) not in {int(c[u]) for u in nb}
        assert set(range(int(c[v]))) <= earlier


def test_greedy_characterisation_random():
    for seed in range(20):
        g = gg.er(60, 1 + seed % 9, seed)
        c, k = oracle.greedy(g)
        _first_fit_characterisation(g, c)
        assert k == c.max() + 1 <= g.max_degree + 1


# ---------------------------------------------------------------------------------------------
# deterministic speculative coloring (Algorithm 1, one vertex per partition)

def _rank(seed, n):
    return oracle.priority_rank(seed, n)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 25])
@pytest.mark.parametrize("seed", [0, 7, 99])
def test_det_complete_graph_closed_form(n, seed):
    # K_n: in round r every worklist vertex sees colors 0..r-2 and takes r-1; only the smallest
    # key keeps it.  So the vertex of key rank k gets color k, and there are n rounds with
    # worklists of sizes n, n-1, ..., 1.
    r = oracle.det(gg.complete(n), seed)
    assert r.rounds == n and r.ncolors == n
    assert np.array_equal(r.colors, _rank(seed, n))
    assert list(r.wl_size) == list(range(n, 0, -1))


@pytest.mark.parametrize("leaves", [1, 2, 5, 40])
@pytest.mark.parametrize("seed", range(6))
def test_det_star_closed_form(leaves, seed):
    # Star with centre 0.  Round 1 colors everything 0.  If the centre has the smallest key it
    # keeps 0 and every leaf takes 1 in round 2 (2 rounds).  Otherwise the centre takes 1 in round
    # 2 (its leaves still show 0); leaves with larger key than the centre also re-take 1 (the
    # centre showed 0), lose to the centre, and take 0 in round 3.  Final: centre 1, leaves 0.
    g = gg.star(leaves)
    rank = _rank(seed, g.n)
    r = oracle.det(g, seed)
    if rank[0] == 0:
        assert r.colors[0] == 0 and np.all(r.colors[1:] == 1) and r.rounds == 2
    else:
        assert r.colors[0] == 1 and np.all(r.colors[1:] == 0)
        assert r.rounds == (3 if np.any(rank[1:] > rank[0]) else 2)


@pytest.mark.parametrize("a,b", [(1, 1), (2, 3), (5, 5), (7, 2), (12, 9)])
@pytest.mark.parametrize("seed", range(8))
def test_det_complete_bipartite_closed_form(a, b, seed):
    # K_{a,b}, sides A = 0..a-1, B = a..a+b-1.  Let S be the side holding the smallest key and T
    # the other side, t = smallest key in T.  Round 1: all 0; all of T loses, and S' = {s in S with
    # key > t} loses.  Round 2: everyone on the worklist sees only 0s and takes 1; every vertex of
    # S' then loses to t.  If S' is empty that ends it (2 rounds, S = 0, T = 1).  Otherwise let
    # s' = smallest key in S'; T'' = {x in T with key > s'} lose too.  Round 3: S' sees T at 1 and
    # takes 0; T'' sees S at {0 (kept), 1 (S' in round 2)} and takes 2.  No conflicts remain.
    edges = [(i, a + j) for i in range(a) for j in range(b)]
    g = gg.from_edges(a + b, edges)
    rank = _rank(seed, a + b)
    A, B = np.arange(a), np.arange(a, a + b)
    S, T = (A, B) if rank[A].min() < rank[B].min() else (B, A)
    t = rank[T].min()
    S1 = S[rank[S] > t]
    r = oracle.det(g, seed)
    if len(S1) == 0:
        assert r.rounds == 2 and np.all(r.colors[S] == 0) and np.all(r.colors[T] == 1)
    else:
        s1 = rank[S1].min()
        T2 = T[rank[T] > s1]
        T1 = T[rank[T] < s1]
        assert r.rounds == 3
        assert np.all(r.colors[S] == 0)
        assert np.all(r.colors[T1] == 1) and np.all(r.colors[T2] == 2)
        assert r.ncolors == (3 if len(T2) else 2)


def test_det_single_edge_and_edgeless():
    for seed in range(5):
        r = oracle.det(gg.path(2), seed)
        rank = _rank(seed, 2)
        assert list(r.colors) == [int(rank[0]), int(rank[1])] and r.rounds == 2
    r = oracle.det(gg.empty(9), 3)
    assert np.all(r.colors == 0) and r.rounds == 1 and r.ncolors == 1
    r = oracle.det(gg.empty(0), 3)
    assert r.rounds == 0 and r.ncolors == 0


def _check_det_invariants(g, seed):
    r = oracle.det(g, seed)
    assert r.status == 0
    c = r.colors
    # Lemma 1: proper at termination
    assert oracle.count_conflicts(g, c) == 0
    if g.n == 0:
        return r
    deg = g.degrees()
    # First Fit never exceeds the degree, hence at most Delta + 1 colors (Section 2.1)
    assert np.all(c >= 0) and np.all(c <= deg)
    assert r.ncolors <= g.max_degree + 1
    assert r.ncolors == len(np.unique(c))
    # a color c can first be taken in round c + 1 (round r sees colors <= r - 2)
    assert r.rounds >= c.max() + 1
    # the smallest key never loses, so it keeps the color 0 of round 1
    rank = _rank(seed, g.n)
    assert c[int(np.argmin(rank))] == 0
    # every round retires the smallest key of its worklist: sizes strictly decrease (rounds <= n)
    assert r.wl_size[0] == g.n and r.wl_degsum[0] == g.nnz
    assert np.all(np.diff(r.wl_size) < 0)
    assert r.rounds <= g.n
    # last_round is consistent with the worklist sizes
    for k in range(r.rounds):
        assert (r.last_round >= k + 1).sum() == r.wl_size[k]
    return r


@pytest.mark.parametrize("seed", range(12))
def test_det_invariants_random(seed):
    _check_det_invariants(gg.er(300, 2 + seed, seed), seed * 31 + 1)
    _check_det_invariants(gg.rmat(9, 8, seed), seed)


def test_det_invariants_structured():
    for g in (gg.stencil27(6), gg.grid5(20, 11), gg.crown(15), gg.cycle(51), gg.workload("er10k")):
        _check_det_invariants(g, 7)


# ---------------------------------------------------------------------------------------------
# brute force on tiny graphs

def _chromatic_number(n, edges):
    if n == 0:
        return 0
    for k in range(1, n + 1):
        for assign in itertools.product(range(k), repeat=n):
            if all(assign[u] != assign[v] for u, v in edges):
                return k
    return n


def _literal_rounds(n, adj, key):
    """Algorithm 1 with one vertex per partition, written directly from Section 3.1 for tiny graphs:
    phase 1 reads the colors of the previous round, phase 2 re-queues the larger key."""
    color = [-1] * n
    work = list(range(n))
    rounds = 0
    while work:
        rounds += 1
        before = list(color)
        for v in work:
            taken = {before[u] for u in adj[v]}
            color[v] = next(c for c in itertools.count() if c not in taken)
        work = [v for v in work if any(color[u] == color[v] and key(u) < key(v) for u in adj[v])]
    return color, rounds


def test_tiny_graphs_brute_force():
    rng = np.random.default_rng(5)
    for trial in range(150):
        n = int(rng.integers(1, 8))
        p = rng.random()
        edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
        g = gg.from_edges(n, edges)
        chi = _chromatic_number(n, edges)
        seed = int(rng.integers(0, 2**63))
        r = oracle.det(g, seed)
        gc_, gk = oracle.greedy(g)
        dmax = g.max_degree
        assert chi <= gk <= dmax + 1
        assert chi <= r.ncolors <= dmax + 1
        adj = [list(g.colidx[g.rowptr[v]:g.rowptr[v + 1]]) for v in range(n)]
        h = oracle.keys(seed, n)
        lit, lr = _literal_rounds(n, adj, lambda v: (int(h[v]), v))
        assert list(r.colors) == lit and r.rounds == lr


# ---------------------------------------------------------------------------------------------
# Algorithm 1 with p id-ordered blocks (Lemma 2 setting)

def test_partition_single_block_is_greedy():
    for seed in range(6):
        g = gg.er(200, 6, seed)
        r = oracle.partition(g, 1)
        c, k = oracle.greedy(g)
        assert np.array_equal(r.colors, c) and r.rounds == 1


@pytest.mark.parametrize("p", [2, 3, 8, 64])
def test_partition_lemma2_round_bound(p):
    # Lemma 2 and its corollary: at most p+1 rounds (block V_p is final after round 1, V_{p-1}
    # after round 2, ...); our reading re-queues the lower block, giving at most p rounds
    for seed in range(10):
        g = gg.er(400, 3 + seed, seed)
        r = oracle.partition(g, p)
        assert r.status == 0
        assert r.rounds <= p <= p + 1
        assert oracle.count_conflicts(g, r.colors) == 0
        assert np.all(r.colors <= g.degrees())


def _literal_alg1(n, adj, p):
    """Algorithm 1 (Section 3.1) restated with its own data structures: blocks V_1..V_p of
    consecutive ids; every vertex keeps ForbiddenColors, one slot per neighbour initialised to -1.
    Phase 1: each block takes its worklist U_i in id order, gives v the least color of
    TotalColors = {0..m} not in v's slots, and writes that color into the slot of v at each
    neighbour in the same block.  Barrier.  Phase 2: each worklist vertex refreshes the slots of its
    neighbours in other blocks and is kept for the next round when one of them in a higher block
    has its color (the reading that the lower block's vertex is recolored).  Barrier.  Returns
    (colors, rounds)."""
    block = [0] * n
    for i in range(p):
        for v in range(i * n // p, (i + 1) * n // p):
            block[v] = i
    m = max((len(a) for a in adj), default=0)
    color = [-1] * n
    forbidden = [{u: -1 for u in adj[v]} for v in range(n)]
    U = [[v for v in range(n) if block[v] == i] for i in range(p)]
    rounds = 0
    while any(U):
        rounds += 1
        for i in range(p):  # phase 1 (threads are independent: only in-block slots are written)
            for v in U[i]:
                used = set(forbidden[v].values())
                color[v] = min(c for c in range(m + 1) if c not in used)
                for u in adj[v]:
                    if block[u] == i:
                        forbidden[u][v] = color[v]
        R = [set() for _ in range(p)]
        for i in range(p):  # phase 2
            for v in U[i]:
                for u in adj[v]:
                    if block[u] != i:
                        forbidden[v][u] = color[u]
                        if color[u] == color[v] and block[u] > i:
                            R[i].add(v)
        U = [sorted(r) for r in R]
    return color, rounds


def test_partition_matches_literal_algorithm1_for_every_block_count():
    # 1 < p < n included: in-block colors seen live, other blocks' colors as refreshed in phase 2
    rng = np.random.default_rng(17)
    for trial in range(80):
        n = int(rng.integers(2, 14))
        dens = float(rng.uniform(0.15, 0.8))
        edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < dens]
        g = gg.from_edges(n, edges)
        adj = [list(g.colidx[g.rowptr[v]:g.rowptr[v + 1]]) for v in range(n)]
        for p in range(1, n + 1):
            lit, lr = _literal_alg1(n, adj, p)
            r = oracle.partition(g, p)
            assert r.status == 0
            assert list(r.colors) == lit and r.rounds == lr, (n, p, edges)


def test_partition_one_vertex_blocks_match_id_priority():
    # p = n: block order = id order, the lower id is re-queued, i.e. the larger id keeps its color
    rng = np.random.default_rng(9)
    for trial in range(60):
        n = int(rng.integers(1, 9))
        edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.5]
        g = gg.from_edges(n, edges)
        adj = [list(g.colidx[g.rowptr[v]:g.rowptr[v + 1]]) for v in range(n)]
        lit, lr = _literal_rounds(n, adj, lambda v: -v)
        r = oracle.partition(g, n)
        assert list(r.colors) == lit and r.rounds == lr


def test_checkers():
    g = gg.complete(4)
    assert oracle.count_conflicts(g, np.array([0, 1, 2, 3], np.int32)) == 0
    assert oracle.count_conflicts(g, np.array([0, 0, 2, 3], np.int32)) == 2
    assert oracle.distinct_colors(np.array([5, 0, 5, 2], np.int32)) == 3


# ---------------------------------------------------------------------------------------------
# largest-first priority (an ordering the paper leaves to future work, Section 6)

def test_lf_key_order():
    rng = np.random.default_rng(13)
    cap = (1 << 20) - 1
    for _ in range(300):
        seed = int(rng.integers(0, 2**63))
        u, v = (int(x) for x in rng.integers(0, 10**6, 2))
        du, dv = (int(x) for x in rng.integers(0, 40, 2))
        want = du > dv if du != dv else oracle.key_less(seed, u, v)
        assert oracle.key_less_lf(seed, u, v, du, dv) == want
    # degrees at or above the cap tie, and the hash decides
    assert oracle.key_less_lf(3, 5, 9, cap + 7, cap) == oracle.key_less(3, 5, 9)
    assert oracle.key_less_lf(3, 9, 5, 2 * cap, cap + 1) == oracle.key_less(3, 9, 5)


@pytest.mark.parametrize("leaves", [1, 2, 31, 500])
def test_lf_star_closed_form(leaves):
    # round 1: everyone 0; the centre has the largest degree and keeps 0, every leaf is re-queued
    # and takes 1 in round 2 (its only neighbour has 0); two colors, two rounds, for any seed
    g = gg.star(leaves)
    deg = g.degrees()
    centre = int(np.argmax(deg))
    for seed in (0, 7):
        r = oracle.det(g, seed, priority=oracle.PRIORITY_LARGEST_FIRST)
        want = np.ones(g.n, np.int32)
        want[centre] = 0
        if leaves == 1:  # two vertices of degree 1: the hash decides who keeps 0
            assert sorted(r.colors) == [0, 1]
        else:
            np.testing.assert_array_equal(r.colors, want)
        assert r.rounds == 2 and r.ncolors == 2


def test_lf_equals_hash_order_on_regular_graphs():
    # equal degrees everywhere: the largest-first key reduces to the hash key
    for g in (gg.cycle(1000), gg.complete(30), gg.crown(20), gg.cycle(7)):
        for seed in (1, 7):
            a = oracle.det(g, seed)
            b = oracle.det(g, seed, priority=oracle.PRIORITY_LARGEST_FIRST)
            np.testing.assert_array_equal(a.colors, b.colors)
            assert (a.rounds, a.ncolors) == (b.rounds, b.ncolors)


def test_lf_tiny_graphs_brute_force():
    rng = np.random.default_rng(17)
    for trial in range(150):
        n = int(rng.integers(1, 8))
        p = rng.random()
        edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
        g = gg.from_edges(n, edges)
        seed = int(rng.integers(0, 2**63))
        r = oracle.det(g, seed, priority=oracle.PRIORITY_LARGEST_FIRST)
        adj = [list(g.colidx[g.rowptr[v]:g.rowptr[v + 1]]) for v in range(n)]
        h = oracle.keys(seed, n)
        deg = g.degrees()
        lit, lr = _literal_rounds(n, adj, lambda v: (-int(deg[v]), int(h[v]), v))
        assert list(r.colors) == lit and r.rounds == lr
        assert _chromatic_number(n, edges) <= r.ncolors <= g.max_degree + 1


# ---------------------------------------------------------------------------------------------
# First Fit in key order (what the ordered mode computes)

def _literal_keyorder(g, key):
    n = g.n
    adj = [list(g.colidx[g.rowptr[v]:g.rowptr[v + 1]]) for v in range(n)]
    color = [-1] * n
    for v in sorted(range(n), key=key):
        taken = {color[u] for u in adj[v]}
        color[v] = next(c for c in itertools.count() if c not in taken)
    return color


def test_keyorder_matches_literal_restatement():
    rng = np.random.default_rng(23)
    for trial in range(40):
        n = int(rng.integers(1, 60))
        edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.2]
        g = gg.from_edges(n, edges)
        seed = int(rng.integers(0, 2**63))
        h = oracle.keys(seed, n)
        deg = g.degrees()
        c, k = oracle.greedy_keyorder(g, seed)
        assert list(c) == _literal_keyorder(g, lambda v: (int(h[v]), v))
        c, k = oracle.greedy_keyorder(g, seed, oracle.PRIORITY_LARGEST_FIRST)
        assert list(c) == _literal_keyorder(g, lambda v: (-int(deg[v]), int(h[v]), v))
        assert k == max(c) + 1


@pytest.mark.parametrize("n", [1, 2, 9, 40])
def test_keyorder_complete_graph(n):
    # in key order every vertex sees all earlier ones colored: rank k gets color k
    g = gg.complete(n)
    for seed in (0, 7):
        c, k = oracle.greedy_keyorder(g, seed)
        np.testing.assert_array_equal(c, _rank(seed, n))
        assert k == n


def test_keyorder_largest_first_welsh_powell_bound():
    # Welsh & Powell (1967): First Fit in non-increasing degree order uses at most
    # max_i min(d_i + 1, i) colors, d_1 >= d_2 >= ... the degrees, i 1-based
    for g in (gg.rmat(12, 8, 1), gg.er(3000, 10.0, 2), gg.star(500), gg.crown(30), gg.grid5(30, 20)):
        c, k = oracle.greedy_keyorder(g, 7, oracle.PRIORITY_LARGEST_FIRST)
        d = np.sort(g.degrees())[::-1]
        bound = int(np.max(np.minimum(d + 1, np.arange(1, g.n + 1))))
        assert k <= bound
        assert oracle.count_conflicts(g, c) == 0 and np.all(c <= g.degrees())


# rounds of the ordered mode: a vertex goes in the round after its last smaller-key neighbour

def _longest_increasing_paths(g, key):
    # every path whose keys increase along it, enumerated from each start; best[v] = the most
    # vertices on such a path ending at v (increasing keys make every such walk a simple path)
    n = g.n
    adj = [list(g.colidx[g.rowptr[v]:g.rowptr[v + 1]]) for v in range(n)]
    best = [0] * n

    def walk(v, length):
        best[v] = max(best[v], length)
        for u in adj[v]:
            if key(u) > key(v):
                walk(u, length + 1)

    for s in range(n):
        if adj[s]:
            walk(s, 1)
    return best


def test_keyorder_depth_brute_force():
    rng = np.random.default_rng(31)
    for trial in range(60):
        n = int(rng.integers(1, 11))
        edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.35]
        g = gg.from_edges(n, edges)
        seed = int(rng.integers(0, 2**63))
        h = oracle.keys(seed, n)
        deg = g.degrees()
        for prio, key in ((oracle.PRIORITY_HASH, lambda v: (int(h[v]), v)),
                          (oracle.PRIORITY_LARGEST_FIRST, lambda v: (-int(deg[v]), int(h[v]), v))):
            depth, k = oracle.keyorder_depth(g, seed, prio)
            assert list(depth) == _longest_increasing_paths(g, key)
            assert k == max([0] + list(depth))


@pytest.mark.parametrize("n", [1, 2, 9, 40])
def test_keyorder_depth_complete_graph(n):
    # the keys form one chain: rank k goes in round k + 1 (a lone vertex is isolated: round 0)
    depth, k = oracle.keyorder_depth(gg.complete(n), 7)
    if n == 1:
        assert list(depth) == [0] and k == 0
    else:
        np.testing.assert_array_equal(depth, _rank(7, n) + 1)
        assert k == n


@pytest.mark.parametrize("leaves", [1, 5, 300])
def test_keyorder_depth_star(leaves):
    # leaves below the center go in round 1, the center next (round 1 if there are none), and the
    # leaves above it in the round after the center
    g = gg.star(leaves)
    h = oracle.keys(7, leaves + 1)
    depth, k = oracle.keyorder_depth(g, 7)
    above = [(int(h[0]), 0) < (int(h[v]), v) for v in range(1, leaves + 1)]
    c = 1 if all(above) else 2
    assert depth[0] == c
    for v in range(1, leaves + 1):
        assert depth[v] == (c + 1 if above[v - 1] else 1)
    assert k == (c + 1 if any(above) else c)


def test_keyorder_depth_edgeless():
    depth, k = oracle.keyorder_depth(gg.empty(17), 7)
    assert not depth.any() and k == 0


# recoloring pass (iterated greedy): First Fit over the classes of a given coloring, largest first

def _recolor_key(h, c):
    return lambda v: (-int(c[v]), int(h[v]), v)


def test_recolor_matches_literal_restatement():
    # any non-negative labels (proper or not) only decide the order
    rng = np.random.default_rng(41)
    for trial in range(40):
        n = int(rng.integers(1, 60))
        edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.2]
        g = gg.from_edges(n, edges)
        seed = int(rng.integers(0, 2**63))
        cin = rng.integers(0, 6, size=n).astype(np.int32)
        c, k = oracle.greedy_keyorder(g, seed, oracle.PRIORITY_RECOLOR, cin)
        assert list(c) == _literal_keyorder(g, _recolor_key(oracle.keys(seed, n), cin))
        depth, _ = oracle.keyorder_depth(g, seed, oracle.PRIORITY_RECOLOR, cin)
        assert list(depth) == _longest_increasing_paths(g, _recolor_key(oracle.keys(seed, n), cin))


def _culberson_check(g, cin, seed):
    # Culberson (1992): with the classes of a proper coloring taken one after another, a vertex of
    # the i-th nonempty class (0-based, largest color first) gets a color <= i
    c, k = oracle.greedy_keyorder(g, seed, oracle.PRIORITY_RECOLOR, cin)
    classes = np.unique(cin)[::-1]
    pos = {int(x): i for i, x in enumerate(classes)}
    assert all(c[v] <= pos[int(cin[v])] for v in range(g.n))
    assert oracle.count_conflicts(g, c) == 0
    assert oracle.distinct_colors(c) <= len(classes)
    return c


def test_recolor_culberson_bound():
    rng = np.random.default_rng(43)
    for g in (gg.rmat(11, 8, 1), gg.er(2000, 12.0, 3), gg.grid5(30, 17), gg.crown(25), gg.stencil27(5)):
        starts = [oracle.greedy(g)[0], oracle.det(g, 7).colors]
        perm = rng.permutation(g.max_degree + 1).astype(np.int32)
        starts.append(3 * perm[oracle.greedy(g)[0]])  # relabelled, with gaps
        for cin in starts:
            c = np.asarray(cin, dtype=np.int32)
            counts = []
            for it in range(4):  # repeated passes never use more colors
                c = _culberson_check(g, c, 11 + it)
                counts.append(oracle.distinct_colors(c))
            assert counts == sorted(counts, reverse=True)
            assert counts[0] <= oracle.distinct_colors(np.asarray(cin))


@pytest.mark.parametrize("n", [2, 9, 40])
def test_recolor_complete_graph_reverses(n):
    # K_n with n distinct colors: the classes are single vertices, taken largest color first
    cin = _rank(7, n).astype(np.int32)
    c, k = oracle.greedy_keyorder(gg.complete(n), 3, oracle.PRIORITY_RECOLOR, cin)
    np.testing.assert_array_equal(c, n - 1 - cin)
    depth, d = oracle.keyorder_depth(gg.complete(n), 3, oracle.PRIORITY_RECOLOR, cin)
    np.testing.assert_array_equal(depth, n - cin)


def test_recolor_keeps_two_colorings():
    for g in (gg.cycle(40), gg.grid5(11, 13), gg.crown(12, interleaved=False)):
        cin = np.asarray(oracle.greedy(g)[0], dtype=np.int32)
        if oracle.distinct_colors(cin) != 2:
            continue
        c, k = oracle.greedy_keyorder(g, 5, oracle.PRIORITY_RECOLOR, cin)
        assert k == 2 and oracle.count_conflicts(g, c) == 0
        np.testing.assert_array_equal(c, 1 - cin)  # class 1 first takes color 0


# smallest-last order by batch peeling

def _degeneracy_matula_beck(g):
    # Matula & Beck (1983): remove a vertex of least remaining degree, one at a time; the
    # degeneracy is the largest degree seen at removal
    n = g.n
    adj = [set(int(u) for u in g.colidx[g.rowptr[v]:g.rowptr[v + 1]]) for v in range(n)]
    deg = {v: len(adj[v]) for v in range(n)}
    best = 0
    while deg:
        v = min(deg, key=lambda x: (deg[x], x))
        best = max(best, deg[v])
        for u in adj[v]:
            if u in deg:
                deg[u] -= 1
        del deg[v]
    return best


def _check_peel_invariant(g, level, k):
    # a vertex was removed with at most k neighbours still present (those removed in its own batch
    # or later), and the levels are 1, 2, ... without gaps
    for v in range(g.n):
        nb = g.colidx[g.rowptr[v]:g.rowptr[v + 1]]
        assert int(np.sum(level[nb] >= level[v])) <= k
    if g.n:
        assert set(np.unique(level)) == set(range(1, int(level.max()) + 1))


def test_peel_degeneracy_brute_force():
    rng = np.random.default_rng(47)
    for trial in range(40):
        n = int(rng.integers(1, 70))
        p = float(rng.choice([0.05, 0.15, 0.4]))
        edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
        g = gg.from_edges(n, edges)
        level, k = oracle.peel_levels(g)
        assert k == _degeneracy_matula_beck(g)
        _check_peel_invariant(g, level, k)
    for g in (gg.rmat(10, 8, 1), gg.grid5(20, 13), gg.stencil27(4)):
        level, k = oracle.peel_levels(g)
        assert k == _degeneracy_matula_beck(g)
        _check_peel_invariant(g, level, k)


@pytest.mark.parametrize("n", [2, 3, 8, 9, 50])
def test_peel_path_closed_form(n):
    # the two ends go first, then the new ends: level = distance to the nearer end + 1
    level, k = oracle.peel_levels(gg.path(n))
    v = np.arange(n)
    np.testing.assert_array_equal(level, np.minimum(v, n - 1 - v) + 1)
    assert k == 1


def test_peel_star_cycle_complete_edgeless():
    level, k = oracle.peel_levels(gg.star(30))
    assert level[0] == 2 and np.all(level[1:] == 1) and k == 1
    level, k = oracle.peel_levels(gg.cycle(25))
    assert np.all(level == 1) and k == 2
    level, k = oracle.peel_levels(gg.complete(12))
    assert np.all(level == 1) and k == 11
    level, k = oracle.peel_levels(gg.empty(9))
    assert np.all(level == 1) and k == 0


def test_smallest_last_greedy_degeneracy_bound():
    # in the smallest-last order a vertex has at most k already-colored neighbours, so First Fit
    # uses at most degeneracy + 1 colors (a bound the natural and hash orders do not have)
    for g in (gg.rmat(12, 8, 1), gg.er(2000, 12.0, 3), gg.grid5(30, 17), gg.stencil27(5), gg.path(40),
              gg.star(100), gg.crown(20)):
        _, k = oracle.peel_levels(g)
        c, nc = oracle.greedy_keyorder(g, 7, oracle.PRIORITY_SMALLEST_LAST)
        assert nc <= k + 1 and oracle.count_conflicts(g, c) == 0
        level, _ = oracle.peel_levels(g)
        h = oracle.keys(7, g.n)
        if g.n <= 300:
            assert list(c) == _literal_keyorder(g, lambda v: (-int(level[v]), int(h[v]), v))


def test_smallest_last_trees_two_colors():
    rng = np.random.default_rng(53)
    for trial in range(10):
        n = int(rng.integers(2, 300))
        edges = [(int(rng.integers(0, i)), i) for i in range(1, n)]  # a random tree
        g = gg.from_edges(n, edges)
        _, k = oracle.peel_levels(g)
        assert k == 1
        c, nc = oracle.greedy_keyorder(g, 3, oracle.PRIORITY_SMALLEST_LAST)
        assert nc == 2 and oracle.count_conflicts(g, c) == 0
        d = oracle.det(g, 3, priority=oracle.PRIORITY_SMALLEST_LAST)
        assert d.status == 0 and oracle.count_conflicts(g, d.colors) == 0
