"""Benchmark: full deterministic speculative coloring of the R-MAT scale-22 graph on one GB300.

One step = one gc_color call on a device-resident CSR (binning, every round, color counting), the
paper's timing convention (Section 5.1: partitioning included, input reading excluded).  Prints one
JSON line.  `--impl reference` times the CPU oracle instead (the reference arm).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat22|stencil256|er10k]
                    [--mode det|inplace|ordered|recolor] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
from math import log as math_log

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gedges/s full coloring on 1 GB300, batched vs one-by-one; colors vs greedy"
HASH_SEED = 7
WORKLOAD_DESC = {
    "rmat22": "R-MAT scale 22 (4,194,304 vertices, edge factor 16, a=.57 b=.19 c=.19 d=.05, seed 2), symmetrised, "
              "deduplicated, self-loops dropped, ids permuted; int32 CSR",
    "stencil256": "3-D 27-point stencil 256^3 (16,777,216 vertices), natural ids; int32 CSR",
    "er10k": "Erdos-Renyi n=10,000 average degree 16, seed 1; int32 CSR",
}
REF_SAMPLE = {  # the reference arm's per-step sample: a few seconds each, so --steps 10 ends in minutes
    "rmat22": ("rmat20", "R-MAT scale 20 (1,048,576 vertices), same recipe, full deterministic coloring"),
    "stencil256": ("stencil128", "27-point stencil 128^3, full deterministic coloring"),
    "er10k": ("er10k", "the same ER graph, full deterministic coloring"),
}

CPU_SAMPLE = {  # bounded oracle sample of the same workload family (10-30 s single-threaded)
    "rmat22": ("rmat21", "R-MAT scale 21 (2,097,152 vertices), same recipe, full deterministic coloring"),
    "stencil256": ("stencil128", "27-point stencil 128^3, full deterministic coloring"),
    "er10k": ("er10k", "the same ER graph, full deterministic coloring"),
}


def algorithmic_bytes(mode, n, wl_size, wl_degsum):
    """Algorithmic bytes of one coloring's round kernel, from the per-round worklist sizes |W_r| and
    degree sums (the ordered modes: per depth).  Deterministic (one fused sweep per round): per
    worklist vertex 4 deg(v) of adjacency + 8 row offsets + 4 worklist entry + 4 own color + 4 color
    write, plus 4 per vertex appended to the next worklist.  In-place: two sweeps per round.
    Ordered and recoloring: the counting pass and the vertex's round each read the row once (row
    offsets, own state, adjacency, one state gather per entry: 16 + 12 deg bytes), plus the count
    write, the ready-list entry and the color (20 bytes a vertex) and an 8-byte count update per
    edge; the recoloring pass also reads the given coloring."""
    E = int(sum(int(x) for x in wl_degsum))  # sum over rounds of sum_{v in W_r} deg(v)
    WT = int(sum(int(x) for x in wl_size))
    if mode == "det":
        return 4 * E + 20 * WT + 4 * (WT - n)
    if mode == "inplace":
        return 2 * (4 * E + 16 * WT) + 4 * (WT - n)
    b = 2 * (12 * E + 16 * WT) + 20 * WT + 8 * (E // 2)
    return b + 4 * n if mode == "recolor" else b


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs (started
    before the warm-up; mark() drops the samples taken before the timed region)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def wait_first_sample(self, timeout_s=5.0):
        t0 = time.perf_counter()
        while self.proc and not self.rows and time.perf_counter() - t0 < timeout_s:
            time.sleep(0.01)

    def mark(self):
        self.rows = []

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def kernel_source_sha256():
    """Digest of the library's sources (the DRAM record applies only to the sources it was taken on)."""
    from paper_1509_08267_gb300._build import source_sha256
    return source_sha256()


def recorded_traffic(workload, mode):
    """DRAM bytes per launch of the round kernel from the committed ncu record for this workload, or
    None when there is none or it was taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", f"round_kernel_{workload}_{mode}_dram.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_sha256") != kernel_source_sha256():
        return None
    return int(rec["dram_bytes_read"]) + int(rec["dram_bytes_write"])


def write_round_table(path, workload, mode, st, rounds, kernel_ms):
    """Per-round table of one statistics run (GC_FLAG_STATS: |W_r|, the degree sum, the entries read
    and the round's duration from its end timestamps; the timestamps add ~0.5 ms to the run)."""
    rn = st.round_ns[:rounds] / 1e3
    lines = [f"# Per round: {mode} coloring of {workload} ({rounds} rounds; {kernel_ms:.2f} ms of kernels "
             "with statistics on)", "",
             "| Rounds | us | entries read | worklist at the first | G entries/s |", "|---|---|---|---|---|"]
    edges = [0, 1, 3, 14, 15, 30, 100, 200, 270, rounds]
    for a, b in zip(edges[:-1], edges[1:]):
        if a >= min(b, rounds):
            continue
        us, rd = rn[a:b].sum(), int(st.round_reads[a:b].sum())
        lines.append(f"| {a + 1}-{min(b, rounds)} | {us:.1f} | {rd} | {int(st.wl_size[a])} | "
                     f"{rd / max(us, 1e-9) / 1e3:.1f} |")
    lines += ["", "| Round | us | worklist | degree sum | entries read |", "|---|---|---|---|---|"]
    for r in range(rounds):
        lines.append(f"| {r + 1} | {rn[r]:.1f} | {int(st.wl_size[r])} | {int(st.wl_degsum[r])} | "
                     f"{int(st.round_reads[r])} |")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def reduce_max(value, world, device=None):
    """The largest of the ranks' values (timing is taken as the slowest rank's); the value itself on
    one rank.  device: where the reduction tensor lives (the rank's GPU under NCCL, CPU under gloo)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_max, world):
    """Whole-job throughput of `world` replicas that each processed units_per_rank units, timed by
    the slowest rank."""
    return world * units_per_rank / seconds_max


def cpu_cores_used():
    return 1  # the oracle is single-threaded


def run_reference(args, rank, world):
    """CPU oracle on the host cores: the reference arm."""
    if rank != 0:
        return
    import graphgen as gg
    import oracle
    key, desc = REF_SAMPLE.get(args.workload, (args.workload, "the same graph, full deterministic coloring"))
    g = gg.workload(key)
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up effects worth a full run; warm-up steps are skipped
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.det(g, HASH_SEED)
        times.append(time.perf_counter() - t0)
        assert r.status == 0
    t = sum(times) / len(times)
    val = (g.nnz / 2) / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Gedges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "sample": desc, "mode": "deterministic"},
        "cpu_baseline": {"value": val, "unit": "Gedges/s", "cores": cpu_cores_used(), "kind": "oracle", "sample": desc},
        "e2e": {"value": val, "unit": "Gedges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_graphs(name):
    """batchG: G graphs of the mixed batch recipe (seed 3), cached on disk."""
    import graphgen as gg
    G = int(name[5:])
    path = os.path.join(gg.cache_dir(), f"{name}_s3.npz")
    if os.path.exists(path):
        z = np.load(path)
        return gg.Batch(G, z["vtx_off"], z["edge_off"], z["rowptr"], z["colidx"])
    b = gg.batch_mix(G, 3)
    if b.colidx.nbytes < (2 << 30):  # large batches are cheaper to regenerate than to cache
        tmp = path + f".tmp{os.getpid()}.npz"
        np.savez(tmp, vtx_off=b.vtx_off, edge_off=b.edge_off, rowptr=b.rowptr, colidx=b.colidx)
        os.replace(tmp, path)
    return b


def shard_graphs(b, rank, world):
    """Graph-sharded batching: the ids (increasing) of the batch's graphs that rank `rank` of
    `world` colors, balanced by vertices + adjacency entries (paper_1509_08267_gb300.dist)."""
    from paper_1509_08267_gb300 import dist as gdist
    sizes = [int(b.edge_off[g + 1] - b.edge_off[g]) + int(b.vtx_off[g + 1] - b.vtx_off[g]) for g in range(b.G)]
    return [g for g, o in enumerate(gdist.shard_graphs(sizes, world)) if o == rank]


def batched_object(args, rank, world, G):
    """Batched coloring of G mixed graphs in one persistent launch against a loop of gc_color over the
    same device-resident graphs, both timed by wall clock around synchronised device work; both must
    give identical colorings.  With several ranks each colors its share of the graphs (no
    collective; the slowest rank's time counts)."""
    import torch

    import graphgen as gg
    import paper_1509_08267_gb300 as gc
    from paper_1509_08267_gb300 import autotune
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    full = batch_graphs(f"batch{G}")
    mine = shard_graphs(full, rank, world) if world > 1 else list(range(full.G))
    b = gg.pack([full.graph(g) for g in mine]) if world > 1 else full
    vo = torch.from_numpy(b.vtx_off).to(dev)
    eo = torch.from_numpy(b.edge_off).to(dev)
    rp = torch.from_numpy(b.rowptr).to(dev)
    ci = torch.from_numpy(b.colidx).to(dev)
    N, NNZ = int(b.vtx_off[-1]), int(b.edge_off[-1])
    out = torch.empty(max(N, 1), dtype=torch.int32, device=dev)[:N]
    tuned = autotune.batch_options()
    steps = max(1, min(args.steps, 5))
    for _ in range(2):
        gc.color_batch(vo, eo, rp, ci, "det", HASH_SEED, out=out, options=tuned)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        _, nc_b, rd_b = gc.color_batch(vo, eo, rp, ci, "det", HASH_SEED, out=out, options=tuned)
    torch.cuda.synchronize()
    t_batch = reduce_max((time.perf_counter() - t0) / steps, world, dev)
    solo = torch.zeros_like(out)  # written once here: no first-touch cost inside the timed loop
    vo_h, eo_h = b.vtx_off, b.edge_off
    nc_s = np.zeros(b.G, np.int32)
    rd_s = np.zeros(b.G, np.int32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g in range(b.G):
        v0, v1, e0, e1 = int(vo_h[g]), int(vo_h[g + 1]), int(eo_h[g]), int(eo_h[g + 1])
        r = gc.color(rp[v0 + g: v1 + g + 1], ci[e0:e1], "det", HASH_SEED, out=solo[v0:v1])
        nc_s[g], rd_s[g] = r.ncolors, r.rounds
    torch.cuda.synchronize()
    t_solo = reduce_max(time.perf_counter() - t0, world, dev)
    same = bool(torch.equal(out, solo)) and np.array_equal(nc_s, nc_b) and np.array_equal(rd_s, rd_b)
    m_job = float(full.edge_off[-1]) / 2  # the whole batch over all ranks
    return {
        "graphs": full.G, "vertices": int(full.vtx_off[-1]), "nnz": int(full.edge_off[-1]),
        "recipe": "n log-uniform [100, 2e5]; even graphs ER (avg degree U[4,64]), odd graphs R-MAT "
                  "(edge factor U[8,16]); seed 3; deterministic mode, hash seed 7",
        "value": m_job / t_batch / 1e9, "unit": "Gedges/s", "ms_per_batch": t_batch * 1e3,
        "one_by_one": {"value": m_job / t_solo / 1e9, "unit": "Gedges/s", "seconds": t_solo,
                       "note": "loop of gc_color over the same device-resident graphs"},
        "batched_over_one_by_one": t_solo / t_batch,
        "identical_colorings": same,
        "timing": "wall clock around synchronised device work, both arms",
        "sharding": f"graphs split over {world} ranks by adjacency entries" if world > 1 else "single",
        "tuned_options": {k: v for k, v in tuned.__dict__.items() if v},
    }


def run_batch(args, rank, world):
    """The batched workload alone (--workload batchG): one JSON line."""
    G = int(args.workload[5:])
    obj = batched_object(args, rank, world, G)
    if rank == 0:
        line = {
            "metric": METRIC, "value": obj["value"], "unit": "Gedges/s", "n_gpus": world,
            "steps": max(1, min(args.steps, 5)), "warmup": args.warmup, "ms_per_step": obj["ms_per_batch"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "graphs": obj["graphs"], "vertices": obj["vertices"],
                       "nnz": obj["nnz"], "recipe": obj["recipe"], "mode": "det", "hash_seed": HASH_SEED,
                       "parallelism": obj["sharding"]},
            "batched": obj,
        }
        print(json.dumps(line), flush=True)


def serve_pool(count, seed=4):
    """Request graphs for the serving benchmark: n log-uniform in [1e3, 2e6], a mix of ER (avg degree
    U[4,32]), R-MAT (edge factor U[4,16]) and 2-D 5-point grids, from the stream `seed` (generated
    on all host cores; the generator releases the GIL)."""
    import math
    from concurrent.futures import ThreadPoolExecutor

    import graphgen as gg
    specs = []
    lo, hi = math.log(1e3), math.log(2e6)
    for i in range(count):
        u0 = (gg.draw(seed, 4 * i) >> 11) / 9007199254740992.0
        u1 = (gg.draw(seed, 4 * i + 1) >> 11) / 9007199254740992.0
        n = int(round(math.exp(lo + u0 * (hi - lo))))
        kind = ("er", "rmat", "grid")[i % 3]
        param = 4 + u1 * 28 if kind == "er" else 4 + u1 * 12
        specs.append(gg.BatchSpec(kind, n, param, gg.draw(seed, 4 * i + 2)))
    with ThreadPoolExecutor(max(1, os.cpu_count() or 1)) as ex:
        return list(ex.map(gg.make_from_spec, specs))


def served_object(args, rank, world, count):
    """Poisson request stream (mean 2,000 req/s, seed 4) into the continuous-batching server, the
    same requests submitted all at once (the server saturated), the same requests colored one by one
    with gc_color (host CSR in, colors out, as the server takes them), and the same graphs as one
    device-resident batch.  Deterministic results must be identical.  With several ranks each runs
    its own server on every world-th request."""
    import torch

    import graphgen as gg
    import paper_1509_08267_gb300 as gc
    from paper_1509_08267_gb300 import autotune
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(local)
    pool = serve_pool(count)
    idx = list(range(rank, count, world))
    graphs = []
    for i in idx:  # the replayed requests sit in pinned host memory, as a server's receive buffers would
        g = pool[i]
        graphs.append(gg.Graph(g.n, torch.from_numpy(g.rowptr).pin_memory().numpy(),
                               torch.from_numpy(g.colidx).pin_memory().numpy(), g.name))
    del pool
    rate = 2000.0
    gaps = [-math_log(1.0 - ((gg.draw(4, 10_000_000 + i) >> 11) / 9007199254740992.0)) / rate for i in idx]
    pv = sum(g.n for g in graphs) + 1
    pe = sum(g.nnz for g in graphs) + 1
    # a bounded pool (a larger one that admits the whole replay at once measured 6% more throughput
    # at twice the p50 and p99 latency)
    pool_v = min(pv, 16_000_000)
    pool_e = min(pe, 600_000_000)
    m_mine = sum(g.nnz for g in graphs) / 2

    def replay(srv, arrivals):
        t0 = time.perf_counter()
        ids = []
        at = 0.0
        for g, gap in zip(graphs, arrivals):
            at += gap
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            ids.append(srv.submit(g.rowptr, g.colidx, mode="det", seed=HASH_SEED))
        res = [srv.poll(rid) for rid in ids]
        return time.perf_counter() - t0, res

    with gc.Server(pool_vertices=pool_v, pool_entries=pool_e, mode="det", seed=HASH_SEED, device=local) as srv:
        replay(srv, [0.0] * min(3, len(graphs)))  # warm-up (allocations, module load)
        t_serve, results = replay(srv, gaps)
        st = srv.stats()
    with gc.Server(pool_vertices=pool_v, pool_entries=pool_e, mode="det", seed=HASH_SEED, device=local) as srv:
        t_sat, results_sat = replay(srv, [0.0] * len(graphs))
    # one by one (host CSR in, colors out, as the server takes them); the library's staging buffers
    # are grown first on the largest request, and the comparisons run after the timed loop
    big = max(range(len(graphs)), key=lambda i: graphs[i].nnz)
    gc.color(graphs[big].rowptr, graphs[big].colidx, "det", HASH_SEED)
    t1 = time.perf_counter()
    solo_res = [gc.color(g.rowptr, g.colidx, "det", HASH_SEED) for g in graphs]
    t_solo = time.perf_counter() - t1
    same = True
    for i, r in enumerate(solo_res):
        for res in (results[i], results_sat[i]):
            same &= bool(np.array_equal(r.colors, res[0])) and r.ncolors == res[1] and r.rounds == res[2]
    del solo_res
    # the same requests as one batch already on the device: co-scheduling all of them at once, with
    # no arrivals to wait for and no copies (an upper bound for the server)
    b = gg.pack(graphs)
    bargs = [torch.from_numpy(a).to(dev) for a in (b.vtx_off, b.edge_off, b.rowptr, b.colidx)]
    bout = torch.empty(int(b.vtx_off[-1]), dtype=torch.int32, device=dev)
    bopt = autotune.batch_options()
    gc.color_batch(*bargs, "det", HASH_SEED, out=bout, options=bopt)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    gc.color_batch(*bargs, "det", HASH_SEED, out=bout, options=bopt)
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t2
    del bargs, bout
    # the same batch from pinned host buffers through one gc_color_batch call (the library stages the
    # CSR to the device and the colors back): the all-at-once bound with the copies a server also makes
    hargs = [torch.from_numpy(a).pin_memory().numpy() for a in (b.vtx_off, b.edge_off, b.rowptr, b.colidx)]
    hout = torch.empty(int(b.vtx_off[-1]), dtype=torch.int32).pin_memory().numpy()
    gc.color_batch(*hargs, "det", HASH_SEED, out=hout, options=bopt)
    t3 = time.perf_counter()
    gc.color_batch(*hargs, "det", HASH_SEED, out=hout, options=bopt)
    t_all_h = time.perf_counter() - t3
    del hargs, hout
    t_serve = reduce_max(t_serve, world, dev)
    t_sat = reduce_max(t_sat, world, dev)
    t_solo = reduce_max(t_solo, world, dev)
    t_all = reduce_max(t_all, world, dev)
    t_all_h = reduce_max(t_all_h, world, dev)
    window = sum(gaps)
    m_job = m_mine * world  # shares are about equal; the slowest rank's time counts
    return {
        "requests": count, "arrival": "Poisson, mean 2,000 req/s, seed 4",
        "graphs": "n log-uniform [1e3, 2e6]; ER / R-MAT / 2-D grid mix", "host_buffers": "pinned",
        "value": m_job / t_serve / 1e9, "unit": "Gedges/s", "graphs_per_s": count / t_serve,
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "serve_wall_s": t_serve,
        "arrival_window_s": window,
        "offered_load_bound": {"value": m_job / max(window, 1e-9) / 1e9, "unit": "Gedges/s",
                               "note": "edges / arrival window: no server can finish before its last request "
                                       "arrives"},
        "saturated": {"value": m_job / t_sat / 1e9, "unit": "Gedges/s", "seconds": t_sat,
                      "note": "every request submitted at once: the server's own capacity"},
        "one_by_one": {"value": m_job / t_solo / 1e9, "unit": "Gedges/s", "graphs_per_s": count / t_solo},
        "served_over_one_by_one": t_solo / t_serve, "saturated_over_one_by_one": t_solo / t_sat,
        "all_at_once": {"value": m_job / t_all / 1e9, "unit": "Gedges/s", "seconds": t_all,
                        "note": "the same graphs as one device-resident gc_color_batch call"},
        "saturated_over_all_at_once": t_all / t_sat,
        "all_at_once_host": {"value": m_job / t_all_h / 1e9, "unit": "Gedges/s", "seconds": t_all_h,
                             "note": "the same batch in one gc_color_batch call from pinned host buffers "
                                     "(CSR staged in, colors out)"},
        "saturated_over_all_at_once_host": t_all_h / t_sat,
        "identical_colorings": same, "rounds_run": st["rounds_run"],
        "pool_vertices": pool_v, "pool_entries": pool_e,
    }


def run_serve(args, rank, world):
    """The serving workload alone (--workload serve): one JSON line."""
    obj = served_object(args, rank, world, args.requests)
    if rank == 0:
        line = {
            "metric": METRIC, "value": obj["value"], "unit": "Gedges/s", "n_gpus": world, "steps": args.requests,
            "warmup": 0, "ms_per_step": obj["serve_wall_s"] * 1e3 / args.requests, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "serve", "requests": args.requests, "arrival": obj["arrival"],
                       "graphs": obj["graphs"], "mode": "det"},
            "served": obj,
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat22", help="rmat22 | stencil256 | er10k | rmatNN | stencilL")
    ap.add_argument("--mode", default="det", choices=["det", "inplace", "ordered", "recolor"])
    ap.add_argument("--priority", default="hash", choices=["hash", "lf", "sl"],
                    help="priority key: seeded hash (default), largest degree first, or smallest last")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--requests", type=int, default=200, help="serving workload: requests replayed")
    ap.add_argument("--batch-graphs", type=int, default=256,
                    help="graphs of the batched object of the default line (0: leave it out)")
    ap.add_argument("--no-served", action="store_true", help="leave the served object out of the default line")
    ap.add_argument("--round-stats", default=None,
                    help="write the per-round table of the warm-up's statistics run to this file")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    import graphgen as gg
    import paper_1509_08267_gb300 as gc

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload.startswith("batch"):
        run_batch(args, rank, world)
        if world > 1:
            dist.destroy_process_group()
        return
    if args.workload == "serve":
        run_serve(args, rank, world)
        if world > 1:
            dist.destroy_process_group()
        return

    gc.load()
    g = gg.workload(args.workload)
    dev = torch.device("cuda", local)
    rp = torch.from_numpy(g.rowptr).to(dev)
    ci = torch.from_numpy(g.colidx).to(dev)
    out = torch.empty(g.n, dtype=torch.int32, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    # first touch outside the timed region: the first write of fresh device pages cost ~250 ms once
    flush.fill_(0)
    prio = {"hash": gc.PRIORITY_HASH, "lf": gc.PRIORITY_LARGEST_FIRST, "sl": gc.PRIORITY_SMALLEST_LAST}[args.priority]
    mode = args.mode
    # the autotuner's options for this graph's class when its table is current, else the defaults
    from paper_1509_08267_gb300 import autotune
    base, tuned_class = autotune.options_for_graph(g.rowptr) if mode in ("det", "inplace") else (gc.Options(), None)
    base.priority = prio
    opt = gc.Options(**{**base.__dict__, "flags": base.flags | gc.FLAG_TIMING})
    start = None
    if mode == "recolor":
        # one recoloring pass over the deterministic mode's coloring (made outside the timed region)
        start = gc.color(rp, ci, "det", HASH_SEED, options=gc.Options(priority=prio))
        start_h = start.colors.cpu().numpy()

    def run(rp_, ci_, out_, **kw):
        if mode == "recolor":
            cin = start.colors if getattr(rp_, "is_cuda", False) else start_h
            return gc.recolor(rp_, ci_, cin, HASH_SEED + 1, out=out_, **kw)
        return gc.color(rp_, ci_, mode, HASH_SEED, out=out_, **kw)

    # the clock sampler starts before the warm-up: nvidia-smi's start-up (NVML initialisation) stays
    # out of the timed region
    clocks = ClockSampler(local)
    clocks.start()
    # warm-up (also records the per-round statistics once, outside the timed region)
    r0 = run(rp, ci, out, stats=True, options=base)
    for _ in range(args.warmup - 1):
        run(rp, ci, out, options=opt)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kernel_ms = []
    clocks.wait_first_sample()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)  # L2 flush between timed steps (outside the events)
        ev[k][0].record(stream)
        res = run(rp, ci, out, options=opt, round_cap=1)
        ev[k][1].record(stream)
        kernel_ms.append(res.stats.kernel_ms)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_max = reduce_max(sum(step_ms) / 1e3, world, dev)
    m_und = g.nnz / 2
    value = whole_job_rate(args.steps * m_und, t_max, world) / 1e9
    ms_per_step = t_max / args.steps * 1e3

    # roofline of the dominant kernel (the persistent round kernel): algorithmic bytes per launch
    st = r0.stats
    alg_bytes = algorithmic_bytes(mode, g.n, st.wl_size, st.wl_degsum)
    kms = statistics.median(kernel_ms)
    peak, peak_kind = load_peaks()
    achieved = alg_bytes / (kms / 1e3) / 1e9

    traffic = recorded_traffic(args.workload, mode) if args.priority == "hash" else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "round phase: persistent round kernel, then (deterministic mode) the core phase's "
                          "kernels; CUDA events around both",
                "kernel_ms": kms, "alg_bytes": alg_bytes,
                "alg_bytes_model": "full-row model of one round of Algorithm 1: 4 deg(v) + 20 per worklist vertex "
                                   "per round + 4 per appended vertex"}
    if traffic is not None:
        # the DRAM bytes the kernels actually moved (ncu) over the same time, against the same peak
        roofline["frac_measured_traffic"] = traffic / (kms / 1e3) / 1e9 / peak

    # end to end through the C ABI with host buffers (pinned): H2D of the CSR, D2H of the colors
    e2e = None
    if args.e2e_steps > 0:
        rp_h = torch.from_numpy(g.rowptr).pin_memory()
        ci_h = torch.from_numpy(g.colidx).pin_memory()
        out_h = torch.empty(g.n, dtype=torch.int32).pin_memory()
        run(rp_h.numpy(), ci_h.numpy(), out_h.numpy(), options=base)
        torch.cuda.synchronize()
        te = []
        for k in range(args.e2e_steps):
            flush.fill_(k & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            run(rp_h.numpy(), ci_h.numpy(), out_h.numpy(), options=base)
            te.append(time.perf_counter() - t0)
        e_t = reduce_max(statistics.median(te), world, dev)
        e2e = {"value": whole_job_rate(m_und, e_t, world) / 1e9, "unit": "Gedges/s",
               "h2d_bytes_per_step": int(4 * (g.n + 1) + 4 * g.nnz + (4 * g.n if mode == "recolor" else 0)),
               "d2h_bytes_per_step": int(4 * g.n + 8),
               "ms_per_step": e_t * 1e3}

    # the batched and served workloads of the same metric, bounded to a minute or two (default line)
    default_line = args.workload == "rmat22" and mode == "det" and args.priority == "hash"
    batched = served = None
    if default_line and args.batch_graphs > 0:
        del rp, ci, out
        torch.cuda.empty_cache()
        batched = batched_object(args, rank, world, args.batch_graphs)
    if default_line and not args.no_served:
        torch.cuda.empty_cache()
        served = served_object(args, rank, world, args.requests)

    if rank == 0:
        import oracle
        greedy_colors = oracle.greedy(g)[1]
        cpu = None
        if not args.no_cpu_baseline:
            key, desc = CPU_SAMPLE.get(args.workload, (args.workload, "the same graph, full deterministic coloring"))
            sg = gg.workload(key)
            oprio = {"hash": 0, "lf": 1, "sl": 2}[args.priority]
            if mode in ("ordered", "recolor"):
                # the oracle of these modes: First Fit in key order (for the recoloring pass, over
                # the oracle's deterministic coloring, which is not timed)
                cin = oracle.det(sg, HASH_SEED).colors if mode == "recolor" else None
                what = ("recoloring pass" if mode == "recolor" else "First Fit in key order")
                desc = desc.replace("full deterministic coloring", what)
                t0 = time.perf_counter()
                if mode == "recolor":
                    oracle.greedy_keyorder(sg, HASH_SEED + 1, oracle.PRIORITY_RECOLOR, cin)
                else:
                    oracle.greedy_keyorder(sg, HASH_SEED, oprio)
                tc = time.perf_counter() - t0
                extra = ""
            else:
                t0 = time.perf_counter()
                ro = oracle.det(sg, HASH_SEED, priority=oprio)
                tc = time.perf_counter() - t0
                extra = f", {ro.rounds} rounds"
            cpu = {"value": (sg.nnz / 2) / tc / 1e9, "unit": "Gedges/s", "cores": cpu_cores_used(), "kind": "oracle",
                   "sample": desc + f" ({tc:.1f} s{extra})",
                   "host_cores_available": os.cpu_count()}
        line = {
            "metric": METRIC, "value": value, "unit": "Gedges/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "graph": WORKLOAD_DESC.get(args.workload, g.name), "n": g.n,
                       "nnz": g.nnz,
                       "mode": {"det": "deterministic", "inplace": "in-place"}.get(mode, mode), "hash_seed": HASH_SEED,
                       "priority": {"hash": "hash", "lf": "largest degree first",
                                    "sl": "smallest last (batch peeling)"}[args.priority],
                       "options": f"autotuned ({tuned_class})" if tuned_class else "library defaults",
                       "l2": "flushed between steps (512 MB write) and colidx > L2", "parallelism":
                       "replicas" if world > 1 else "single"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            # setup, degree sort (2), expand, round kernel, color count (2) per coloring, plus the core
            # phase's four (index, fill, core rounds, write-back) and the tail phase's cluster launch in
            # deterministic mode; ordered mode and recoloring: setup, counting pass, round kernel,
            # color count (2) (smallest last adds the peeling's two: its set-up and the peeling kernel)
            "gpu_launches": ((5 if mode in ("ordered", "recolor") else 7) + (5 if mode == "det" else 0)
                             + (2 if args.priority == "sl" else 0)) * args.steps,
            "clocks": clk,
            **({"batched": batched} if batched is not None else {}),
            **({"served": served} if served is not None else {}),
            "rounds": r0.rounds, "ncolors": r0.ncolors, "greedy_ncolors": greedy_colors,
            **({"ncolors_before_recolor": start.ncolors} if start is not None else {}),
            "max_degree": g.max_degree, "wall_s_timed": t_wall,
        }
        print(json.dumps(line), flush=True)
        if args.round_stats and r0.stats is not None:
            write_round_table(args.round_stats, args.workload, mode, r0.stats, r0.rounds, r0.stats.kernel_ms)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
