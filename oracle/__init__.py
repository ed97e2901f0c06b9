"""CPU oracle for speculative first-fit graph coloring (arXiv:1509.08267, Section 3.1, Algorithm 1).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline
(and its ``--impl reference`` arm) import this package.  The CUDA library in
``paper_1509_08267_gb300`` never imports, links or calls it, and the two share no code.

The arithmetic is in ``gc_oracle.c`` (plain single-threaded C, compiled with gcc on first use);
this module only marshals numpy arrays.  Functions:

* ``greedy(g)``            -- sequential First Fit in natural order (Section 3, Section 5).
* ``det(g, seed)``         -- round-by-round deterministic speculative coloring (Algorithm 1 with
                              one vertex per partition and a SplitMix64 hash priority).
* ``partition(g, p)``      -- Algorithm 1 with p id-ordered blocks (Lemma 2's setting).
* ``splitmix64(seed, i)``, ``key_less(seed, u, v)``, ``keys(seed, n)`` -- the priority key.
* ``count_conflicts``, ``distinct_colors`` -- checks used by the tests.

Pins: every function here is checked in ``tests/test_oracle_pins.py`` against facts the paper or
mathematics fixes (published SplitMix64 outputs, closed forms on K_n, stars, cycles, grids, the
27-point stencil and crown graphs, brute-force chromatic numbers, Lemma 1 and Lemma 2, and an
independently written literal-rule simulation on tiny graphs).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_library(force: bool = False) -> str:
    """Compile gc_oracle.c into _build/liboracle.so (single-threaded, -O2)."""
    with _lock:
        src = os.path.join(_HERE, "gc_oracle.c")
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
            return _SO
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        r = subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", tmp],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
        os.replace(tmp, _SO)
        return _SO


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_library())
        i32, i64, u64, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        lib.oracle_splitmix64.restype = u64
        lib.oracle_splitmix64.argtypes = [u64, u64]
        lib.oracle_key_less.restype = ctypes.c_int
        lib.oracle_key_less.argtypes = [u64, i32, i32]
        lib.oracle_keys.restype = None
        lib.oracle_keys.argtypes = [u64, i32, p]
        lib.oracle_distinct_colors.restype = i32
        lib.oracle_distinct_colors.argtypes = [i32, p]
        lib.oracle_count_conflicts.restype = i64
        lib.oracle_count_conflicts.argtypes = [i32, p, p, p]
        lib.oracle_greedy.restype = i32
        lib.oracle_greedy.argtypes = [i32, p, p, p]
        lib.oracle_det.restype = ctypes.c_int
        lib.oracle_det.argtypes = [i32, p, p, u64, i32, p, p, p, p, p, i32, p]
        lib.oracle_det_prio.restype = ctypes.c_int
        lib.oracle_det_prio.argtypes = [i32, p, p, u64, i32, p, i32, p, p, p, p, p, i32, p]
        lib.oracle_greedy_keyorder.restype = i32
        lib.oracle_greedy_keyorder.argtypes = [i32, p, p, u64, i32, p, p]
        lib.oracle_peel_levels.restype = i32
        lib.oracle_peel_levels.argtypes = [i32, p, p, p]
        lib.oracle_keyorder_depth.restype = i32
        lib.oracle_keyorder_depth.argtypes = [i32, p, p, u64, i32, p, p]
        lib.oracle_key_less_lf.restype = ctypes.c_int
        lib.oracle_key_less_lf.argtypes = [u64, i32, i32, i32, i32]
        lib.oracle_partition.restype = ctypes.c_int
        lib.oracle_partition.argtypes = [i32, p, p, i32, i32, p, p, p, p, i32]
        _lib = lib
    return _lib


U64 = (1 << 64) - 1


def _csr(g):
    rp = np.ascontiguousarray(g.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(g.colidx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)
    return rp, ci


def splitmix64(seed: int, index: int) -> int:
    """Output number `index` (0-based) of SplitMix64 seeded with `seed`."""
    return int(_L().oracle_splitmix64(seed & U64, index & U64))


def key_less(seed: int, u: int, v: int) -> bool:
    """True when key(u) < key(v): u keeps its color against v."""
    return bool(_L().oracle_key_less(seed & U64, u, v))


def keys(seed: int, n: int) -> np.ndarray:
    out = np.empty(max(n, 1), dtype=np.uint64)
    _L().oracle_keys(seed & U64, n, out.ctypes.data)
    return out[:n]


def priority_rank(seed: int, n: int) -> np.ndarray:
    """rank[v] = position of v when vertices are sorted by key (0 = keeps its color against all)."""
    h = keys(seed, n)
    order = np.lexsort((np.arange(n), h))
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    return rank


def distinct_colors(colors: np.ndarray) -> int:
    c = np.ascontiguousarray(colors, dtype=np.int32)
    if c.size == 0:
        return 0
    return int(_L().oracle_distinct_colors(c.size, c.ctypes.data))


def count_conflicts(g, colors: np.ndarray) -> int:
    """Directed adjacency entries whose endpoints share a color (0 for a proper coloring)."""
    rp, ci = _csr(g)
    c = np.ascontiguousarray(colors, dtype=np.int32)
    if g.n == 0:
        return 0
    return int(_L().oracle_count_conflicts(g.n, rp.ctypes.data, ci.ctypes.data, c.ctypes.data))


def greedy(g) -> tuple[np.ndarray, int]:
    """Sequential First Fit in natural order: (colors, number of colors)."""
    rp, ci = _csr(g)
    colors = np.empty(max(g.n, 1), dtype=np.int32)
    nc = _L().oracle_greedy(g.n, rp.ctypes.data, ci.ctypes.data, colors.ctypes.data)
    if nc < 0:
        raise MemoryError("oracle_greedy")
    return colors[: g.n], int(nc)


@dataclass
class DetResult:
    colors: np.ndarray
    ncolors: int
    rounds: int
    status: int
    wl_size: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    wl_degsum: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    last_round: np.ndarray | None = None


PRIORITY_HASH = 0
PRIORITY_LARGEST_FIRST = 1
PRIORITY_SMALLEST_LAST = 2  # key (-min(level(v), 2^20 - 1), h(v), v), level from peel_levels
PRIORITY_RECOLOR = 3  # key (-min(c(v), 2^20 - 1), h(v), v) for a given coloring c


def key_less_lf(seed: int, u: int, v: int, du: int, dv: int) -> bool:
    """Largest-first priority: u keeps its color against v (degrees capped at 2^20 - 1, ties by hash)."""
    return bool(_L().oracle_key_less_lf(seed & U64, u, v, du, dv))


def peel_levels(g) -> tuple[np.ndarray, int]:
    """Smallest-last levels by batch peeling (level[v] >= 1 is the batch that removed v; later
    batches are colored first) and the largest threshold reached, the degeneracy."""
    rp, ci = _csr(g)
    level = np.empty(max(g.n, 1), dtype=np.int32)
    k = _L().oracle_peel_levels(g.n, rp.ctypes.data, ci.ctypes.data, level.ctypes.data)
    if k < 0:
        raise MemoryError("oracle_peel_levels")
    return level[:g.n], int(k)


def _colors_in(g, priority, colors_in):
    if priority == PRIORITY_SMALLEST_LAST:
        a = np.ascontiguousarray(peel_levels(g)[0], dtype=np.int32)
        return (a.ctypes.data if a.size else None), a
    if priority != PRIORITY_RECOLOR:
        return None, None
    a = np.ascontiguousarray(colors_in, dtype=np.int32)
    if a.shape != (g.n,) or (g.n and a.min() < 0):
        raise ValueError("colors_in must be int32[n] with entries >= 0")
    return (a.ctypes.data if a.size else None), a


def greedy_keyorder(g, seed: int, priority: int = PRIORITY_HASH, colors_in=None) -> tuple[np.ndarray, int]:
    """Sequential First Fit in increasing key order (the hash key, largest degree first, or, for
    PRIORITY_RECOLOR, the color classes of colors_in with the largest color first)."""
    rp, ci = _csr(g)
    pin, keep = _colors_in(g, priority, colors_in)
    colors = np.empty(max(g.n, 1), dtype=np.int32)
    k = _L().oracle_greedy_keyorder(g.n, rp.ctypes.data, ci.ctypes.data, seed & U64, int(priority), pin,
                                    colors.ctypes.data)
    if k < 0:
        raise MemoryError("oracle_greedy_keyorder")
    return colors[:g.n], int(k)


def keyorder_depth(g, seed: int, priority: int = PRIORITY_HASH, colors_in=None) -> tuple[np.ndarray, int]:
    """Per-vertex round of First Fit in key order when each vertex goes as soon as its smaller-key
    neighbours are colored (0 for isolated vertices), and the largest such round."""
    rp, ci = _csr(g)
    pin, keep = _colors_in(g, priority, colors_in)
    depth = np.empty(max(g.n, 1), dtype=np.int32)
    k = _L().oracle_keyorder_depth(g.n, rp.ctypes.data, ci.ctypes.data, seed & U64, int(priority), pin,
                                   depth.ctypes.data)
    if k < 0:
        raise MemoryError("oracle_keyorder_depth")
    return depth[:g.n], int(k)


def det(g, seed: int, max_rounds: int | None = None, stats_cap: int = 1 << 16,
        priority: int = PRIORITY_HASH) -> DetResult:
    """Deterministic speculative coloring, round by round.  `status` is 0, or -1 when the round
    cap (default n + 1) was reached with a non-empty worklist.  `last_round[v]` is the last round
    whose worklist held v (worklists only shrink, so v was on W_1..W_last_round[v]).  priority:
    PRIORITY_HASH (key = hash, id), PRIORITY_LARGEST_FIRST (key = -capped degree, hash, id) or
    PRIORITY_SMALLEST_LAST (key = -capped peel level, hash, id)."""
    rp, ci = _csr(g)
    n = g.n
    if max_rounds is None:
        max_rounds = n + 1
    cap = max(1, min(stats_cap, max_rounds))
    colors = np.empty(max(n, 1), dtype=np.int32)
    wl = np.zeros(cap, dtype=np.int64)
    ds = np.zeros(cap, dtype=np.int64)
    nc = ctypes.c_int32(0)
    rd = ctypes.c_int32(0)
    last = np.zeros(max(n, 1), dtype=np.int32)
    pin, keep = _colors_in(g, priority, None) if priority == PRIORITY_SMALLEST_LAST else (None, None)
    st = _L().oracle_det_prio(n, rp.ctypes.data, ci.ctypes.data, seed & U64, int(priority), pin, max_rounds,
                              colors.ctypes.data, ctypes.byref(nc), ctypes.byref(rd), wl.ctypes.data, ds.ctypes.data,
                              cap, last.ctypes.data)
    if st == -2:
        raise MemoryError("oracle_det")
    r = int(rd.value)
    k = min(r, cap)
    return DetResult(colors[:n], int(nc.value), r, int(st), wl[:k].copy(), ds[:k].copy(), last[:n])


def partition(g, p: int, max_rounds: int | None = None, stats_cap: int = 1 << 16) -> DetResult:
    """Algorithm 1 with p id-ordered blocks (block priority, sequential first fit inside a block)."""
    rp, ci = _csr(g)
    n = g.n
    if max_rounds is None:
        max_rounds = n + 1
    cap = max(1, min(stats_cap, max_rounds))
    colors = np.empty(max(n, 1), dtype=np.int32)
    wl = np.zeros(cap, dtype=np.int64)
    nc = ctypes.c_int32(0)
    rd = ctypes.c_int32(0)
    st = _L().oracle_partition(n, rp.ctypes.data, ci.ctypes.data, p, max_rounds, colors.ctypes.data,
                               ctypes.byref(nc), ctypes.byref(rd), wl.ctypes.data, cap)
    if st == -2:
        raise MemoryError("oracle_partition")
    r = int(rd.value)
    return DetResult(colors[:n], int(nc.value), r, int(st), wl[: min(r, cap)].copy())
