"""Python binding of libgc.so, the GB300 speculative graph-coloring library (include/gc.h).

Argument marshalling only: every step of the coloring runs in the library's CUDA kernels.  Arrays
may be CUDA tensors (used in place, on the current torch stream) or host arrays (numpy or CPU
tensors, staged by the library).  There is no CPU fallback: if ``libgc.so`` has not been built, or
no CUDA device is usable, every call raises :class:`GCError`.

Method: Singhal, Peri & Kalyanasundaram, arXiv:1509.08267, Section 3.1 (Algorithm 1), with one
vertex per partition and a SplitMix64 priority; see ``include/gc.h`` for the exact contract.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "GCError", "load", "color", "color_batch", "validate", "det_round", "Options", "Stats", "Server", "MODE_DETERMINISTIC",
    "MODE_INPLACE", "MODE_PARTITION", "MODE_ORDERED", "PRIORITY_HASH", "PRIORITY_LARGEST_FIRST", "PRIORITY_SMALLEST_LAST", "smallest_last", "recolor", "version", "release_scratch",
]

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgc.so")

GC_OK = 0
GC_ERR_INVALID_ARG = -1
GC_ERR_INVALID_GRAPH = -2
GC_ERR_OOM = -3
GC_ERR_CUDA = -4
GC_ERR_NO_CONVERGENCE = -5
GC_ERR_TIMEOUT = -6
GC_ERR_BUSY = -7
STATUS_NAMES = {0: "GC_OK", -1: "GC_ERR_INVALID_ARG", -2: "GC_ERR_INVALID_GRAPH", -3: "GC_ERR_OOM",
                -4: "GC_ERR_CUDA", -5: "GC_ERR_NO_CONVERGENCE", -6: "GC_ERR_TIMEOUT", -7: "GC_ERR_BUSY"}

MODE_DETERMINISTIC = 0
MODE_INPLACE = 1
MODE_PARTITION = 2
MODE_ORDERED = 3
PRIORITY_HASH = 0
PRIORITY_LARGEST_FIRST = 1
PRIORITY_SMALLEST_LAST = 2
FLAG_STATS = 1
FLAG_TIMING = 2
FLAG_VALIDATE = 4
FLAG_FULL_SWEEP = 8
VALIDATE_SORTED = 1
VALIDATE_SYMMETRIC = 2
VALIDATE_ALL = 3


class GCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class _Options(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("max_rounds", ctypes.c_int32), ("small_max_degree", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("block_size", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("spin_limit_ns", ctypes.c_int64), ("flags", ctypes.c_uint32), ("partitions", ctypes.c_int32),
                ("priority", ctypes.c_int32), ("core_vertices", ctypes.c_int32),
                ("core_entries", ctypes.c_int32), ("tail_vertices", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class _Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("ncolors", ctypes.c_int32), ("max_color", ctypes.c_int32),
                ("round_cap", ctypes.c_int32), ("wl_size", ctypes.c_void_p), ("wl_degsum", ctypes.c_void_p),
                ("round_ns", ctypes.c_void_p),
                ("worklist_total", ctypes.c_int64), ("entries_scanned", ctypes.c_int64), ("kernel_ms", ctypes.c_float),
                ("setup_ms", ctypes.c_float), ("grid_blocks", ctypes.c_int32), ("block_size", ctypes.c_int32),
                ("round_reads", ctypes.c_void_p), ("reserved", ctypes.c_int32 * 4)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("pool_vertices", ctypes.c_int64), ("pool_entries", ctypes.c_int64),
                ("max_requests", ctypes.c_int32), ("mode", ctypes.c_int32), ("spin_limit_ns", ctypes.c_int64),
                ("device", ctypes.c_int32), ("solo_entries", ctypes.c_int32), ("reserved", ctypes.c_int32 * 6)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("rounds_run", ctypes.c_int64), ("vertices_colored", ctypes.c_int64),
                ("edges_colored", ctypes.c_int64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("wall_s", ctypes.c_double), ("resident", ctypes.c_int32),
                ("queued", ctypes.c_int32), ("failed", ctypes.c_int64), ("reserved", ctypes.c_int32 * 4)]


_lib = None


def load(path: str | None = None):
    """Loads libgc.so (raises GCError when it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise GCError(GC_ERR_CUDA, f"{path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    i32, i64, u64, p, P = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER
    c_int = ctypes.c_int
    lib.gc_color.restype = c_int
    lib.gc_color.argtypes = [i32, p, p, c_int, u64, p, p, p]
    lib.gc_color_ex.restype = c_int
    lib.gc_color_ex.argtypes = [i32, p, p, c_int, u64, p, p, p, P(_Options), P(_Stats)]
    lib.gc_recolor.restype = c_int
    lib.gc_recolor.argtypes = [i32, p, p, p, u64, p, p, p, P(_Options), P(_Stats)]
    lib.gc_smallest_last.restype = c_int
    lib.gc_smallest_last.argtypes = [i32, p, p, p, p, p, P(_Options)]
    lib.gc_color_batch.restype = c_int
    lib.gc_color_batch.argtypes = [i32, p, p, p, p, c_int, u64, p, p, p]
    lib.gc_color_batch_ex.restype = c_int
    lib.gc_color_batch_ex.argtypes = [i32, p, p, p, p, c_int, u64, p, p, p, P(_Options), P(_Stats)]
    lib.gc_validate_graph.restype = c_int
    lib.gc_validate_graph.argtypes = [i32, p, p, c_int]
    lib.gc_last_error.restype = ctypes.c_char_p
    lib.gc_last_error.argtypes = []
    lib.gc_version.restype = c_int
    lib.gc_release_scratch.restype = c_int
    lib.gc_det_round.restype = c_int
    lib.gc_det_round.argtypes = [i32, p, p, u64, p, p, i32, p, p]
    if hasattr(lib, "gc_server_create"):
        lib.gc_server_create.restype = c_int
        lib.gc_server_create.argtypes = [P(_ServerConfig), P(p)]
        lib.gc_server_submit.restype = c_int
        lib.gc_server_submit.argtypes = [p, i32, p, p, c_int, u64, P(u64)]
        lib.gc_server_poll.restype = c_int
        lib.gc_server_poll.argtypes = [p, u64, i32, p, p, p]
        lib.gc_server_stats.restype = c_int
        lib.gc_server_stats.argtypes = [p, P(_ServerStats)]
        lib.gc_server_stats_get.restype = c_int
        lib.gc_server_stats_get.argtypes = [p, P(_ServerStats)]
        lib.gc_server_destroy.restype = None
        lib.gc_server_destroy.argtypes = [p]
    _lib = lib
    return lib


def _check(status: int):
    if status != GC_OK:
        raise GCError(status, load().gc_last_error().decode(errors="replace"))


def version() -> int:
    return int(load().gc_version())


def release_scratch():
    _check(load().gc_release_scratch())


# ---------------------------------------------------------------------------------------------
# marshalling helpers

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """Raw pointer of a contiguous array of the given numpy dtype (numpy, CPU or CUDA tensor)."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        want = {np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if x.dtype != want:
            raise TypeError(f"expected {want}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr() if x.numel() else None, x
    a = np.ascontiguousarray(x, dtype=dtype)
    return (a.ctypes.data if a.size else None), a


def _on_cuda(x) -> bool:
    return _is_torch(x) and x.is_cuda


def _current_stream(*arrays):
    for a in arrays:
        if _on_cuda(a):
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return ctypes.c_void_p(0)


def _empty_like_home(ref, n: int, dtype=np.int32):
    if _on_cuda(ref):
        import torch
        return torch.empty(max(n, 1), dtype={np.int32: torch.int32}[dtype], device=ref.device)[:n]
    return np.empty(n, dtype=dtype)


@dataclass
class Options:
    """Knobs of gc_options (0 = library default)."""
    max_rounds: int = 0
    small_max_degree: int = 0
    chunk: int = 0
    block_size: int = 0
    blocks_per_sm: int = 0
    spin_limit_ns: int = 0
    flags: int = 0
    partitions: int = 0
    priority: int = 0
    core_vertices: int = 0
    core_entries: int = 0
    tail_vertices: int = 0

    def _c(self, stream) -> _Options:
        o = _Options()
        o.stream = stream
        o.max_rounds = self.max_rounds
        o.small_max_degree = self.small_max_degree
        o.chunk = self.chunk
        o.block_size = self.block_size
        o.blocks_per_sm = self.blocks_per_sm
        o.spin_limit_ns = self.spin_limit_ns
        o.flags = self.flags
        o.partitions = self.partitions
        o.priority = self.priority
        o.core_vertices = self.core_vertices
        o.core_entries = self.core_entries
        o.tail_vertices = self.tail_vertices
        return o


@dataclass
class Stats:
    rounds: int = 0
    ncolors: int = 0
    max_color: int = -1
    worklist_total: int = 0
    entries_scanned: int = 0
    kernel_ms: float = 0.0
    setup_ms: float = 0.0
    grid_blocks: int = 0
    block_size: int = 0
    wl_size: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    wl_degsum: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    round_ns: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    round_reads: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))


def _mode(mode) -> int:
    if isinstance(mode, str):
        return {"det": 0, "deterministic": 0, "inplace": 1, "in-place": 1, "partition": 2, "ordered": 3}[mode]
    return int(mode)


@dataclass
class Result:
    colors: object  # int32 array on the inputs' home (CUDA tensor or numpy)
    ncolors: int
    rounds: int
    stats: Stats | None = None


def color(rowptr, colidx, mode="det", seed: int = 0, out=None, options: Options | None = None,
          stats: bool = False, round_cap: int = 1 << 16) -> Result:
    """Colors one graph (gc_color_ex).  rowptr: int32[n+1], colidx: int32[nnz]."""
    return _color_one(rowptr, colidx, mode, seed, out, options, stats, round_cap, None)


def recolor(rowptr, colidx, colors_in, seed: int = 0, out=None, options: Options | None = None,
            stats: bool = False, round_cap: int = 1 << 16) -> Result:
    """One iterated-greedy recoloring pass (gc_recolor): First Fit over the color classes of
    colors_in (int32[n], >= 0), the largest color first; never more colors than colors_in has
    when colors_in is proper."""
    return _color_one(rowptr, colidx, "ordered", seed, out, options, stats, round_cap, colors_in)


def det_round(rowptr, colidx, seed: int, colors_cur, worklist, colors_next=None, lost=None):
    """One deterministic round over the worklist vertices `worklist` (gc_det_round): reading C_r
    (colors_cur, int32[n]) returns (colors_next, lost), int32[len(worklist)] each, on the
    worklist's home (CUDA tensor or numpy)."""
    lib = load()
    n = (rowptr.numel() if _is_torch(rowptr) else len(rowptr)) - 1
    nwork = worklist.numel() if _is_torch(worklist) else len(worklist)
    prp, rk = _ptr(rowptr, np.int32)
    pci, ck = _ptr(colidx, np.int32)
    pcur, curk = _ptr(colors_cur, np.int32)
    pw, wk = _ptr(worklist, np.int32)
    if colors_next is None:
        colors_next = _empty_like_home(worklist, nwork)
    if lost is None:
        lost = _empty_like_home(worklist, nwork)
    pn, nk = _ptr(colors_next, np.int32)
    pl, lk = _ptr(lost, np.int32)
    _check(lib.gc_det_round(n, prp, pci, seed & ((1 << 64) - 1), pcur, pw, nwork, pn, pl))
    return (nk if nk is not None else colors_next), (lk if lk is not None else lost)


def smallest_last(rowptr, colidx, out=None, options: Options | None = None):
    """Smallest-last levels by batch peeling (gc_smallest_last).  Returns (level[n], number of
    levels, degeneracy); level is on the device when rowptr is a CUDA tensor."""
    lib = load()
    n = (rowptr.numel() if _is_torch(rowptr) else len(rowptr)) - 1
    if n < 0:
        raise GCError(GC_ERR_INVALID_ARG, "rowptr must have n+1 entries")
    prp, rowptr_k = _ptr(rowptr, np.int32)
    pci, colidx_k = _ptr(colidx, np.int32)
    if out is None:
        out = _empty_like_home(rowptr, n)
    pout, out_k = _ptr(out, np.int32)
    nl = ctypes.c_int32(0)
    dg = ctypes.c_int32(0)
    copt = (options or Options())._c(_current_stream(rowptr, colidx, out))
    _check(lib.gc_smallest_last(n, prp, pci, pout, ctypes.byref(nl), ctypes.byref(dg), ctypes.byref(copt)))
    return (out_k if out_k is not None else out), int(nl.value), int(dg.value)


def _color_one(rowptr, colidx, mode, seed, out, options, stats, round_cap, colors_in) -> Result:
    lib = load()
    n = (rowptr.numel() if _is_torch(rowptr) else len(rowptr)) - 1
    if n < 0:
        raise GCError(GC_ERR_INVALID_ARG, "rowptr must have n+1 entries")
    prp, rowptr_k = _ptr(rowptr, np.int32)
    pci, colidx_k = _ptr(colidx, np.int32)
    if out is None:
        out = _empty_like_home(rowptr, n)
    pout, out_k = _ptr(out, np.int32)
    nc = ctypes.c_int32(0)
    rd = ctypes.c_int32(0)
    opt = (options or Options())
    if stats:
        opt = Options(**{**opt.__dict__, "flags": opt.flags | FLAG_STATS | FLAG_TIMING})
    want_stats = bool(opt.flags & (FLAG_STATS | FLAG_TIMING))
    copt = opt._c(_current_stream(rowptr, colidx, out))
    st = _Stats()
    wl = np.zeros(round_cap, np.int64)
    ds = np.zeros(round_cap, np.int64)
    rn = np.zeros(round_cap, np.int64)
    rr = np.zeros(round_cap, np.int64)
    st.round_cap = round_cap
    st.wl_size = wl.ctypes.data
    st.wl_degsum = ds.ctypes.data
    st.round_ns = rn.ctypes.data
    st.round_reads = rr.ctypes.data
    if colors_in is None:
        _check(lib.gc_color_ex(n, prp, pci, _mode(mode), seed & ((1 << 64) - 1), pout, ctypes.byref(nc),
                               ctypes.byref(rd), ctypes.byref(copt), ctypes.byref(st)))
    else:
        pin, colors_in_k = _ptr(colors_in, np.int32)
        _check(lib.gc_recolor(n, prp, pci, pin, seed & ((1 << 64) - 1), pout, ctypes.byref(nc),
                              ctypes.byref(rd), ctypes.byref(copt), ctypes.byref(st)))
    s = None
    if want_stats:
        k = min(st.rounds, round_cap)
        s = Stats(st.rounds, st.ncolors, st.max_color, st.worklist_total, st.entries_scanned, st.kernel_ms,
                  st.setup_ms, st.grid_blocks, st.block_size, wl[:k].copy(), ds[:k].copy(), rn[:k].copy(),
                  rr[:k].copy())
    return Result(out_k if out_k is not None else out, int(nc.value), int(rd.value), s)


def color_batch(vtx_off, edge_off, rowptr, colidx, mode="det", seed: int = 0, out=None,
                options: Options | None = None, stats: bool = False, round_cap: int = 1 << 16):
    """Colors G packed graphs in one launch (gc_color_batch_ex).  Returns (colors, ncolors[G], rounds[G]
    [, Stats]) with per-graph arrays as numpy (Stats covers the whole batch, per round)."""
    lib = load()
    G = (vtx_off.numel() if _is_torch(vtx_off) else len(vtx_off)) - 1
    N = int(vtx_off[-1])
    pv, vk = _ptr(vtx_off, np.int64)
    pe, ek = _ptr(edge_off, np.int64)
    prp, rk = _ptr(rowptr, np.int32)
    pci, ck = _ptr(colidx, np.int32)
    if out is None:
        out = _empty_like_home(rowptr, N)
    pout, ok = _ptr(out, np.int32)
    nc = np.zeros(max(G, 1), np.int32)
    rd = np.zeros(max(G, 1), np.int32)
    opt = (options or Options())
    if stats:
        opt = Options(**{**opt.__dict__, "flags": opt.flags | FLAG_STATS | FLAG_TIMING})
    copt = opt._c(_current_stream(vtx_off, rowptr, colidx, out))
    st = _Stats()
    wl = np.zeros(round_cap, np.int64)
    ds = np.zeros(round_cap, np.int64)
    rn = np.zeros(round_cap, np.int64)
    rr = np.zeros(round_cap, np.int64)
    st.round_cap = round_cap
    st.wl_size = wl.ctypes.data
    st.wl_degsum = ds.ctypes.data
    st.round_ns = rn.ctypes.data
    st.round_reads = rr.ctypes.data
    _check(lib.gc_color_batch_ex(G, pv, pe, prp, pci, _mode(mode), seed & ((1 << 64) - 1), pout, nc.ctypes.data,
                                 rd.ctypes.data, ctypes.byref(copt), ctypes.byref(st)))
    res = (ok if ok is not None else out, nc[:G], rd[:G])
    if stats:
        k = min(st.rounds, round_cap)
        res = res + (Stats(st.rounds, st.ncolors, st.max_color, st.worklist_total, st.entries_scanned, st.kernel_ms,
                           st.setup_ms, st.grid_blocks, st.block_size, wl[:k].copy(), ds[:k].copy(),
                           rn[:k].copy(), rr[:k].copy()),)
    return res


def validate(rowptr, colidx, flags: int = VALIDATE_ALL) -> None:
    """Raises GCError(GC_ERR_INVALID_GRAPH) when the CSR breaks the graph format."""
    lib = load()
    n = (rowptr.numel() if _is_torch(rowptr) else len(rowptr)) - 1
    prp, rk = _ptr(rowptr, np.int32)
    pci, ck = _ptr(colidx, np.int32)
    _check(lib.gc_validate_graph(n, prp, pci, flags))


class Server:
    """Continuous-batching coloring server (gc_server_*).  `mode` and `seed` are the defaults of
    submit(); the pool of `mode` is allocated with the server, the other mode's at its first
    request."""

    def __init__(self, pool_vertices: int, pool_entries: int, max_requests: int = 0, mode="det", seed: int = 0,
                 device: int = -1, spin_limit_ns: int = 0, solo_entries: int = 0):
        lib = load()
        cfg = _ServerConfig()
        cfg.pool_vertices = pool_vertices
        cfg.pool_entries = pool_entries
        cfg.max_requests = max_requests
        cfg.mode = _mode(mode)
        cfg.spin_limit_ns = spin_limit_ns
        cfg.device = device
        cfg.solo_entries = solo_entries
        h = ctypes.c_void_p()
        _check(lib.gc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._n = {}
        self._mode = mode
        self._seed = seed

    def submit(self, rowptr, colidx, mode=None, seed: int | None = None) -> int:
        """Queues one graph with its own mode and priority seed (the server's defaults if None)."""
        n = (rowptr.numel() if _is_torch(rowptr) else len(rowptr)) - 1
        prp, rk = _ptr(rowptr, np.int32)
        pci, ck = _ptr(colidx, np.int32)
        rid = ctypes.c_uint64(0)
        m = _mode(self._mode if mode is None else mode)
        sd = (self._seed if seed is None else seed) & ((1 << 64) - 1)
        _check(load().gc_server_submit(self._h, n, prp, pci, m, sd, ctypes.byref(rid)))
        self._n[rid.value] = n
        return int(rid.value)

    def poll(self, req_id: int, timeout_ms: int = -1, out=None):
        """Returns (colors, ncolors, rounds) when done, None while pending (GC_ERR_BUSY)."""
        n = self._n[req_id]
        if out is None:
            out = np.empty(n, np.int32)
        pout, ok = _ptr(out, np.int32)
        nc = ctypes.c_int32(0)
        rd = ctypes.c_int32(0)
        st = load().gc_server_poll(self._h, req_id, timeout_ms, pout, ctypes.byref(nc), ctypes.byref(rd))
        if st == GC_ERR_BUSY:
            return None
        self._n.pop(req_id, None)
        _check(st)
        return (ok if ok is not None else out), int(nc.value), int(rd.value)

    def stats(self) -> dict:
        s = _ServerStats()
        _check(load().gc_server_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in _ServerStats._fields_ if k != "reserved"}

    def close(self):
        if self._h:
            load().gc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
