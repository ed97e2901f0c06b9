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
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

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
    """Digest of the round kernel's sources (the kernels and the layout constants they use)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("gc_kernels.cu", "gc_internal.h"):
        with open(os.path.join(ROOT, "paper_1509_08267_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


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


def run_batch(args, rank, world):
    """Batched coloring of G graphs in one persistent launch against a loop of gc_color over the same
    device-resident graphs; both must give identical colorings."""
    import torch
    import torch.distributed as dist

    import paper_1509_08267_gb300 as gc
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    b = batch_graphs(args.workload)
    G = b.G
    vo = torch.from_numpy(b.vtx_off).to(dev)
    eo = torch.from_numpy(b.edge_off).to(dev)
    rp = torch.from_numpy(b.rowptr).to(dev)
    ci = torch.from_numpy(b.colidx).to(dev)
    N, NNZ = int(b.vtx_off[-1]), int(b.edge_off[-1])
    out = torch.empty(N, dtype=torch.int32, device=dev)
    from paper_1509_08267_gb300 import autotune
    tuned = autotune.batch_options()  # knobs chosen by the autotuner for batches (defaults without a table)
    opt = gc.Options(**{**tuned.__dict__, "flags": tuned.flags | gc.FLAG_TIMING})
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        gc.color_batch(vo, eo, rp, ci, args.mode, HASH_SEED, out=out, options=opt)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    clocks.start()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        _, nc_b, rd_b, st = gc.color_batch(vo, eo, rp, ci, args.mode, HASH_SEED, out=out, options=opt, stats=True)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_batch = reduce_max(sum(a.elapsed_time(c) for a, c in ev) / 1e3 / args.steps, world, dev)
    # one by one: the same device-resident graphs, one gc_color call each (each call synchronises)
    solo = torch.empty(N, dtype=torch.int32, device=dev)
    vo_h, eo_h = b.vtx_off, b.edge_off
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nc_s = np.zeros(G, np.int32)
    rd_s = np.zeros(G, np.int32)
    for g in range(G):
        v0, v1, e0, e1 = int(vo_h[g]), int(vo_h[g + 1]), int(eo_h[g]), int(eo_h[g + 1])
        r = gc.color(rp[v0 + g: v1 + g + 1], ci[e0:e1], args.mode, HASH_SEED, out=solo[v0:v1])
        nc_s[g], rd_s[g] = r.ncolors, r.rounds
    torch.cuda.synchronize()
    t_solo = time.perf_counter() - t0
    same = bool(torch.equal(out, solo)) and np.array_equal(nc_s, nc_b) and np.array_equal(rd_s, rd_b)
    m_und = NNZ / 2
    if rank == 0:
        line = {
            "metric": METRIC, "value": whole_job_rate(m_und, t_batch, world) / 1e9, "unit": "Gedges/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "graphs": G, "vertices": N, "nnz": NNZ,
                       "recipe": "n log-uniform [100, 2e5]; even graphs ER (avg degree U[4,64]), odd graphs R-MAT "
                                 "(edge factor U[8,16]); seed 3", "mode": args.mode, "hash_seed": HASH_SEED},
            "one_by_one": {"value": m_und / t_solo / 1e9, "unit": "Gedges/s", "seconds": t_solo,
                           "note": "loop of gc_color over the same device-resident graphs"},
            "batched_over_one_by_one": t_solo / t_batch,
            "identical_colorings": same,
            "batch_rounds": int(st.rounds), "batch_kernel_ms": st.kernel_ms,
            "tuned_options": {k: v for k, v in tuned.__dict__.items() if v},
            # batch tables, setup, degree sort (2), expand, round kernel, color count (2) per call
            "gpu_launches": 8 * args.steps, "clocks": clk,
        }
        print(json.dumps(line), flush=True)


def serve_pool(count, seed=4):
    """Request graphs for the serving benchmark: n log-uniform in [1e3, 2e6], a mix of ER (avg degree
    U[4,32]), R-MAT (edge factor U[4,16]) and 2-D 5-point grids, from the stream `seed`."""
    import math

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
    return [gg.make_from_spec(s) for s in specs]


def run_serve(args, rank, world):
    """Poisson request stream into the continuous-batching server against the same requests colored
    one by one with gc_color; results must be identical."""
    import torch

    import paper_1509_08267_gb300 as gc
    import graphgen as gg
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    count = args.requests
    # the replayed requests sit in pinned host memory, as a server's receive buffers would
    graphs = []
    for g in serve_pool(count):
        rp = torch.from_numpy(g.rowptr).pin_memory().numpy()
        ci = torch.from_numpy(g.colidx).pin_memory().numpy()
        graphs.append(gg.Graph(g.n, rp, ci, g.name))
    rate = 2000.0
    gaps = [-math_log(1.0 - ((gg.draw(4, 10_000_000 + i) >> 11) / 9007199254740992.0)) / rate for i in range(count)]
    pv = sum(g.n for g in graphs) + 1
    pe = sum(g.nnz for g in graphs) + 1
    pool_v = min(pv, 16_000_000)
    pool_e = min(pe, 600_000_000)
    results = {}
    with gc.Server(pool_vertices=pool_v, pool_entries=pool_e, mode=args.mode, seed=HASH_SEED, device=local) as srv:
        t0 = time.perf_counter()
        ids = []
        at = 0.0
        for g, gap in zip(graphs, gaps):
            at += gap
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            ids.append(srv.submit(g.rowptr, g.colidx))
        for i, rid in enumerate(ids):
            results[i] = srv.poll(rid)
        t_serve = time.perf_counter() - t0
        st = srv.stats()
    # one by one, host arrays in and out as the server takes them
    t1 = time.perf_counter()
    same = True
    for i, g in enumerate(graphs):
        r = gc.color(g.rowptr, g.colidx, args.mode, HASH_SEED)
        if args.mode == "det":
            same &= bool(np.array_equal(r.colors, results[i][0])) and r.ncolors == results[i][1] and \
                r.rounds == results[i][2]
    t_solo = time.perf_counter() - t1
    dev = torch.device("cuda", local)
    # the same requests as one batch already on the device: what co-scheduling all of them at once
    # gives, with no arrivals to wait for and no copies (an upper bound for the server)
    b = gg.pack(graphs)
    bargs = [torch.from_numpy(a).to(dev) for a in (b.vtx_off, b.edge_off, b.rowptr, b.colidx)]
    bout = torch.empty(int(b.vtx_off[-1]), dtype=torch.int32, device=dev)
    from paper_1509_08267_gb300 import autotune
    bopt = autotune.batch_options()
    gc.color_batch(*bargs, args.mode, HASH_SEED, out=bout, options=bopt)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    gc.color_batch(*bargs, args.mode, HASH_SEED, out=bout, options=bopt)
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t2
    del bargs, bout
    t_serve = reduce_max(t_serve, world, dev)
    t_solo = reduce_max(t_solo, world, dev)
    t_all = reduce_max(t_all, world, dev)
    m_und = sum(g.nnz for g in graphs) / 2
    if rank == 0:
        line = {
            "metric": METRIC, "value": whole_job_rate(m_und, t_serve, world) / 1e9, "unit": "Gedges/s",
            "n_gpus": world, "steps": count,
            "warmup": 0, "ms_per_step": t_serve * 1e3 / count, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "serve", "requests": count, "arrival": "Poisson, mean 2,000 req/s, seed 4",
                       "host_buffers": "pinned",
                       "graphs": "n log-uniform [1e3, 2e6]; ER / R-MAT / 2-D grid mix",
                       "pool_vertices": pool_v, "pool_entries": pool_e, "mode": args.mode},
            "graphs_per_s": count / t_serve, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "one_by_one": {"value": m_und / t_solo / 1e9, "unit": "Gedges/s", "graphs_per_s": count / t_solo},
            "served_over_one_by_one": t_solo / t_serve, "identical_colorings": same,
            "all_at_once": {"value": m_und / t_all / 1e9, "unit": "Gedges/s", "seconds": t_all,
                            "note": "the same graphs as one device-resident gc_color_batch call"},
            "rounds_run": st["rounds_run"], "server_busy_s": st["busy_s"], "serve_wall_s": t_serve,
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
    prio = {"hash": gc.PRIORITY_HASH, "lf": gc.PRIORITY_LARGEST_FIRST, "sl": gc.PRIORITY_SMALLEST_LAST}[args.priority]
    opt = gc.Options(flags=gc.FLAG_TIMING, priority=prio)
    mode = args.mode
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

    # warm-up (also records the per-round statistics once, outside the timed region)
    r0 = run(rp, ci, out, stats=True, options=gc.Options(priority=prio))
    for _ in range(args.warmup - 1):
        run(rp, ci, out, options=opt)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kernel_ms = []
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
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

    # end to end through the C ABI with host buffers (pinned): H2D of the CSR, D2H of the colors
    e2e = None
    if args.e2e_steps > 0:
        rp_h = torch.from_numpy(g.rowptr).pin_memory()
        ci_h = torch.from_numpy(g.colidx).pin_memory()
        out_h = torch.empty(g.n, dtype=torch.int32).pin_memory()
        run(rp_h.numpy(), ci_h.numpy(), out_h.numpy(), options=gc.Options(priority=prio))
        torch.cuda.synchronize()
        te = []
        for k in range(args.e2e_steps):
            flush.fill_(k & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            run(rp_h.numpy(), ci_h.numpy(), out_h.numpy(), options=gc.Options(priority=prio))
            te.append(time.perf_counter() - t0)
        e_t = reduce_max(statistics.median(te), world, dev)
        e2e = {"value": whole_job_rate(m_und, e_t, world) / 1e9, "unit": "Gedges/s",
               "h2d_bytes_per_step": int(4 * (g.n + 1) + 4 * g.nnz + (4 * g.n if mode == "recolor" else 0)),
               "d2h_bytes_per_step": int(4 * g.n + 8),
               "ms_per_step": e_t * 1e3}

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
                       "l2": "flushed between steps (512 MB write) and colidx > L2", "parallelism":
                       "replicas" if world > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": recorded_traffic(args.workload, mode) if args.priority == "hash" else None,
                         "peak_kind": peak_kind,
                         "kernel": "round kernel (persistent)", "kernel_ms": kms, "alg_bytes": alg_bytes},
            "cpu_baseline": cpu,
            "e2e": e2e,
            # setup, degree sort (2), expand, round kernel, color count (2) per coloring; ordered mode
            # and recoloring: setup, counting pass, round kernel, color count (2)
            # (smallest last adds the peeling's two: its set-up and the peeling kernel)
            "gpu_launches": ((5 if mode in ("ordered", "recolor") else 7) + (2 if args.priority == "sl" else 0))
            * args.steps,
            "clocks": clk,
            "rounds": r0.rounds, "ncolors": r0.ncolors, "greedy_ncolors": greedy_colors,
            **({"ncolors_before_recolor": start.ncolors} if start is not None else {}),
            "max_degree": g.max_degree, "wall_s_timed": t_wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
