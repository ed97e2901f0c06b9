"""gc_det_round on the GPU: one round of the deterministic mode over a block's worklist, and the
vertex-block driver (Algorithm 1's partitions V_1..V_p, Section 3.1) built on it, against the
oracle for several block counts."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _dev(g):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(g.rowptr)).cuda(),
            torch.from_numpy(np.ascontiguousarray(g.colidx if g.nnz else np.zeros(1, np.int32))).cuda())


@pytest.mark.parametrize("make", [lambda: gg.rmat(14, 16, 2), lambda: gg.workload("er10k"), lambda: gg.complete(600),
                                  lambda: gg.stencil27(9), lambda: gg.star(3000), lambda: gg.empty(9),
                                  lambda: gg.crown(40)])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_vertex_blocks_on_gpu_match_oracle(gclib, make, world):
    from paper_1509_08267_gb300 import dist as gdist
    g = make()
    rp, ci = _dev(g)
    ref = oracle.det(g, 7)
    colors, rounds = gdist.color_blocks_inprocess(rp, ci, 7, gdist.gpu_step(rp, ci, 7), world)
    np.testing.assert_array_equal(colors.cpu().numpy(), ref.colors)
    assert rounds == ref.rounds


def test_det_round_first_round(gclib):
    # round 1 reads C_1 = 0 everywhere: a vertex loses iff some neighbour has a smaller key, and a
    # loser's next color is 1 (its neighbours all have 0)
    g = gg.rmat(12, 16, 2)
    rank = oracle.priority_rank(3, g.n)
    work = np.flatnonzero(np.diff(g.rowptr) > 0).astype(np.int32)
    nxt, lost = gclib.det_round(g.rowptr, g.colidx, 3, np.zeros(g.n, np.int32), work)
    for i, v in enumerate(work):
        nb = g.colidx[g.rowptr[v]:g.rowptr[v + 1]]
        want = bool((rank[nb] < rank[v]).any())
        assert lost[i] == want
        assert nxt[i] == (1 if want else 0)


def test_det_round_rejects_bad_input(gclib):
    g = gg.cycle(6)
    with pytest.raises(gclib.GCError) as ei:
        gclib.det_round(g.rowptr, g.colidx, 1, np.zeros(6, np.int32), np.array([0, 9], np.int32))
    assert ei.value.status == gclib.GC_ERR_INVALID_ARG
    bad = g.colidx.copy()
    bad[0] = 0  # self-loop on vertex 0
    with pytest.raises(gclib.GCError) as ei:
        gclib.det_round(g.rowptr, bad, 1, np.zeros(6, np.int32), np.arange(6, dtype=np.int32))
    assert ei.value.status == gclib.GC_ERR_INVALID_GRAPH
