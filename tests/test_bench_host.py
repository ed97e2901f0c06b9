"""bench.py's per-round table (--round-stats) from a statistics record, on worklists the oracle
produces (no GPU): every round appears once with its worklist, degree sum and entries read, and the
grouped rows add up to the per-round ones."""
import types

import numpy as np

import bench
import graphgen as gg
import oracle


def test_round_table_rows_and_groups(tmp_path):
    g = gg.rmat(10, 8, 3)
    ref = oracle.det(g, 7)
    R = ref.rounds
    st = types.SimpleNamespace(round_ns=np.arange(1, R + 1, dtype=np.float64) * 1000.0,
                               wl_size=ref.wl_size.astype(np.int64), wl_degsum=ref.wl_degsum.astype(np.int64),
                               round_reads=ref.wl_degsum.astype(np.int64) // 2)
    path = tmp_path / "rounds.md"
    bench.write_round_table(str(path), "rmat10", "det", st, R, 1.25)
    lines = path.read_text().splitlines()
    assert lines[0].startswith("# Per round: det coloring of rmat10") and f"({R} rounds" in lines[0]
    rows = [l.split("|")[1:-1] for l in lines if l.startswith("| ") and l.split("|")[1].strip().isdigit()]
    assert [int(r[0]) for r in rows] == list(range(1, R + 1))
    for r, (_, us, w, ds, rd) in zip(range(R), rows):
        assert float(us) == (r + 1) * 1.0
        assert int(w) == ref.wl_size[r] and int(ds) == ref.wl_degsum[r] and int(rd) == ref.wl_degsum[r] // 2
    groups = [l.split("|")[1:-1] for l in lines if l.startswith("| ") and "-" in l.split("|")[1]
              and l.split("|")[1].strip()[0].isdigit()]
    assert sum(int(x[2]) for x in groups) == int(st.round_reads.sum())
    assert int(groups[-1][0].split("-")[1]) == R
