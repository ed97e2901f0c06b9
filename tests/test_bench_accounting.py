"""The roofline's algorithmic bytes (bench.algorithmic_bytes) against the per-vertex byte model
written out vertex by vertex, on worklists the oracle produces (no GPU)."""
import numpy as np

import bench
import graphgen as gg
import oracle


def _explicit_det(g, ref, inplace=False):
    # deterministic: one fused sweep per round; in-place: assignment and conflict sweeps
    deg = g.degrees()
    total = 0
    last = ref.last_round  # v was on W_1 .. W_last[v]
    for v in range(g.n):
        for r in range(1, int(last[v]) + 1):
            if inplace:
                total += 2 * (4 * int(deg[v]) + 16)
            else:
                total += 4 * int(deg[v]) + 20
            if r >= 2:
                total += 4  # appended to W_r by round r - 1
    return total


def test_det_bytes_match_per_vertex_model():
    for g in (gg.complete(7), gg.star(40), gg.rmat(9, 8, 1), gg.er(500, 6.0, 2)):
        ref = oracle.det(g, 7)
        got = bench.algorithmic_bytes("det", g.n, ref.wl_size, ref.wl_degsum)
        assert got == _explicit_det(g, ref)
        got = bench.algorithmic_bytes("inplace", g.n, ref.wl_size, ref.wl_degsum)
        assert got == _explicit_det(g, ref, inplace=True)


def test_complete_graph_closed_form():
    # K_n: W_r has n - r + 1 vertices of degree n - 1
    n = 9
    ref = oracle.det(gg.complete(n), 3)
    sizes = np.arange(n, 0, -1)
    b = int(np.sum(sizes * (4 * (n - 1) + 20))) + 4 * int(np.sum(sizes[1:]))
    assert bench.algorithmic_bytes("det", n, ref.wl_size, ref.wl_degsum) == b


def test_ordered_bytes_match_per_vertex_model():
    for g in (gg.rmat(9, 8, 1), gg.grid5(20, 17), gg.star(30)):
        depth, deepest = oracle.keyorder_depth(g, 7)
        deg = g.degrees()
        sizes = [int(np.sum(depth == d)) for d in range(1, deepest + 1)]
        sums = [int(deg[depth == d].sum()) for d in range(1, deepest + 1)]
        explicit = 0
        for v in range(g.n):
            if deg[v] == 0:
                continue
            d = int(deg[v])
            explicit += 2 * (16 + 12 * d) + 20  # counting pass + round; count, ready entry, color
        explicit += 8 * (int(deg.sum()) // 2)  # one count update per edge
        assert bench.algorithmic_bytes("ordered", g.n, sizes, sums) == explicit
        assert bench.algorithmic_bytes("recolor", g.n, sizes, sums) == explicit + 4 * g.n
