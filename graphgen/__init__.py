"""Seeded synthetic graph generators shared by the CPU oracle's tests and the CUDA library's tests.

This package is input plumbing only: it builds undirected simple graphs as int32 CSR (rows sorted,
symmetric, no self-loops, no duplicate entries) and holds none of the coloring arithmetic.  The
heavy lifting is in ``graphgen.c`` (plain C, compiled on first use with gcc); this module wraps it
with numpy and caches large graphs as ``.npz`` files.

Workloads (sizes as used by the tests and the benchmark):

* ``er(n, avg_degree, seed)`` -- Erdos-Renyi G(n, M) with M = n*avg_degree/2 uniformly drawn pairs.
* ``rmat(scale, edge_factor, seed)`` -- R-MAT with a, b, c, d = .57, .19, .19, .05, vertex ids
  randomly permuted (the power-law stand-in for the social graphs of the paper's Section 5).
* ``stencil27(L)`` -- 3-D 27-point stencil, natural lexicographic ids.
* ``grid5(Lx, Ly)`` -- 2-D 5-point grid.
* ``batch_mix(G, seed, ...)`` -- many graphs of log-uniform size, half ER and half R-MAT.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

# The permutation stream is offset from the edge stream by a fixed odd constant.
PERM_STREAM_OFFSET = 0x5851F42D4C957F2D
U64 = (1 << 64) - 1


@dataclass
class Graph:
    """An undirected simple graph in int32 CSR form."""

    n: int
    rowptr: np.ndarray  # int32[n+1]
    colidx: np.ndarray  # int32[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1]) if self.n > 0 else 0

    @property
    def m(self) -> int:
        """Number of undirected edges."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr.astype(np.int64))

    @property
    def max_degree(self) -> int:
        return int(self.degrees().max()) if self.n > 0 else 0


def build_library(force: bool = False) -> str:
    """Compile graphgen.c into _build/libgraphgen.so (OpenMP when available)."""
    with _lock:
        src = os.path.join(_HERE, "graphgen.c")
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
            return _SO
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", tmp]
        r = subprocess.run(base[:2] + ["-fopenmp"] + base[2:], capture_output=True, text=True)
        if r.returncode != 0:
            r = subprocess.run(base, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("graphgen build failed:\n" + r.stderr)
        os.replace(tmp, _SO)
        return _SO


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_library())
        i32, i64, u64, dbl, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
        lib.gg_draw.restype = u64
        lib.gg_draw.argtypes = [u64, u64]
        lib.gg_er_pairs.restype = i64
        lib.gg_er_pairs.argtypes = [i32, i64, u64, p, p]
        lib.gg_rmat_pairs.restype = i64
        lib.gg_rmat_pairs.argtypes = [i32, ctypes.c_int, i64, dbl, dbl, dbl, u64, p, p]
        lib.gg_permutation.restype = None
        lib.gg_permutation.argtypes = [i32, u64, p]
        lib.gg_csr_from_pairs.restype = i64
        lib.gg_csr_from_pairs.argtypes = [i32, i64, p, p, p, p, p]
        lib.gg_stencil27_nnz.restype = i64
        lib.gg_stencil27_nnz.argtypes = [i32]
        lib.gg_stencil27.restype = i64
        lib.gg_stencil27.argtypes = [i32, p, p]
        lib.gg_grid5_nnz.restype = i64
        lib.gg_grid5_nnz.argtypes = [i32, i32]
        lib.gg_grid5.restype = i64
        lib.gg_grid5.argtypes = [i32, i32, p, p]
        lib.gg_batch.restype = ctypes.c_int
        lib.gg_batch.argtypes = [i32, p, p, p, p, dbl, dbl, dbl, u64, p, p, p, p, p]
        lib.gg_batch_pack.restype = None
        lib.gg_batch_pack.argtypes = [i32, p, p, p]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def draw(seed: int, k: int) -> int:
    """Draw number k of the SplitMix64 stream seeded with `seed` (generator stream only)."""
    return int(_L().gg_draw(seed & U64, k & U64))


def from_pairs(n: int, src: np.ndarray, dst: np.ndarray, perm: np.ndarray | None = None, name: str = "") -> Graph:
    """Symmetrise, relabel (new id = perm[old]), sort and deduplicate a pair list into CSR."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    M = int(src.shape[0])
    if perm is not None:
        perm = np.ascontiguousarray(perm, dtype=np.int32)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    colidx = np.empty(max(2 * M, 1), dtype=np.int32)
    nnz = _L().gg_csr_from_pairs(n, M, _ptr(src), _ptr(dst), _ptr(perm), _ptr(rowptr), _ptr(colidx))
    if nnz < 0:
        raise ValueError("graph too large for int32 CSR")
    return Graph(n, rowptr, colidx[:nnz].copy(), name)


def from_edges(n: int, edges, name: str = "") -> Graph:
    """CSR from an iterable of undirected (u, v) pairs (small graphs for tests)."""
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    return from_pairs(n, e[:, 0], e[:, 1], name=name)


def _round_half_up(x: float) -> int:
    return int(math.floor(x + 0.5))


def er(n: int, avg_degree: float, seed: int) -> Graph:
    """Erdos-Renyi G(n, M) with M = floor(n * avg_degree / 2 + 1/2) uniform pairs u != v (with replacement)."""
    M = _round_half_up(n * avg_degree / 2)
    src = np.empty(M, dtype=np.int32)
    dst = np.empty(M, dtype=np.int32)
    if _L().gg_er_pairs(n, M, seed & U64, _ptr(src), _ptr(dst)) < 0:
        raise ValueError("bad ER arguments")
    return from_pairs(n, src, dst, name=f"er_n{n}_d{avg_degree:g}_s{seed}")


def permutation(n: int, seed: int) -> np.ndarray:
    perm = np.empty(n, dtype=np.int32)
    _L().gg_permutation(n, (seed + PERM_STREAM_OFFSET) & U64, _ptr(perm))
    return perm


def rmat(scale: int, edge_factor: float, seed: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         n: int | None = None, permute: bool = True) -> Graph:
    """R-MAT with M = round(edge_factor * n) sampled pairs, symmetrised, deduplicated, self-loops
    dropped and (by default) ids permuted by a seeded uniform permutation."""
    if n is None:
        n = 1 << scale
    M = _round_half_up(edge_factor * n)
    src = np.empty(M, dtype=np.int32)
    dst = np.empty(M, dtype=np.int32)
    if _L().gg_rmat_pairs(n, scale, M, a, b, c, seed & U64, _ptr(src), _ptr(dst)) < 0:
        raise ValueError("bad R-MAT arguments")
    perm = permutation(n, seed) if permute else None
    return from_pairs(n, src, dst, perm, name=f"rmat_s{scale}_n{n}_ef{edge_factor:g}_s{seed}")


def stencil27(L: int) -> Graph:
    n = L * L * L
    nnz = int(_L().gg_stencil27_nnz(L))
    rowptr = np.empty(n + 1, dtype=np.int32)
    colidx = np.empty(max(nnz, 1), dtype=np.int32)
    if _L().gg_stencil27(L, _ptr(rowptr), _ptr(colidx)) < 0:
        raise ValueError("stencil too large for int32 CSR")
    return Graph(n, rowptr, colidx[:nnz], name=f"stencil27_L{L}")


def grid5(Lx: int, Ly: int) -> Graph:
    n = Lx * Ly
    nnz = int(_L().gg_grid5_nnz(Lx, Ly))
    rowptr = np.empty(n + 1, dtype=np.int32)
    colidx = np.empty(max(nnz, 1), dtype=np.int32)
    if _L().gg_grid5(Lx, Ly, _ptr(rowptr), _ptr(colidx)) < 0:
        raise ValueError("grid too large for int32 CSR")
    return Graph(n, rowptr, colidx[:nnz], name=f"grid5_{Lx}x{Ly}")


# ---------------------------------------------------------------------------------------------
# small named graphs (tests)

def complete(n: int) -> Graph:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], name=f"K{n}")


def cycle(n: int) -> Graph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], name=f"C{n}")


def path(n: int) -> Graph:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], name=f"P{n}")


def star(leaves: int) -> Graph:
    """Star K_{1,leaves} with centre 0."""
    return from_edges(leaves + 1, [(0, i) for i in range(1, leaves + 1)], name=f"star{leaves}")


def empty(n: int) -> Graph:
    return Graph(n, np.zeros(n + 1, dtype=np.int32), np.zeros(0, dtype=np.int32), name=f"empty{n}")


def crown(k: int, interleaved: bool = True) -> Graph:
    """Crown graph: K_{k,k} minus a perfect matching.  Sides a_i, b_i, edges a_i-b_j for i != j.
    Interleaved ids (a_0, b_0, a_1, b_1, ...) make natural-order first fit use k colors; side
    ids (all a, then all b) make it use 2."""
    def a(i):
        return 2 * i if interleaved else i

    def b(i):
        return 2 * i + 1 if interleaved else k + i

    return from_edges(2 * k, [(a(i), b(j)) for i in range(k) for j in range(k) if i != j],
                      name=f"crown{k}{'i' if interleaved else 's'}")


# ---------------------------------------------------------------------------------------------
# batches

@dataclass
class BatchSpec:
    kind: str  # "er" | "rmat"
    n: int
    param: float  # ER average degree or R-MAT edge factor
    seed: int


def batch_specs(G: int, seed: int, nmin: int = 100, nmax: int = 200_000, er_deg=(4.0, 64.0),
                rmat_ef=(8.0, 16.0)) -> list[BatchSpec]:
    """Per-graph parameters of a mixed batch.  Graph g draws four values from the stream `seed`
    (draws 4g..4g+3): log-uniform n in [nmin, nmax], the degree parameter (uniform in the given
    range), and its own generator seed.  Even g are ER, odd g are R-MAT."""
    specs = []
    lo, hi = math.log(nmin), math.log(nmax)
    for g in range(G):
        u0 = (draw(seed, 4 * g) >> 11) / 9007199254740992.0
        u1 = (draw(seed, 4 * g + 1) >> 11) / 9007199254740992.0
        gseed = draw(seed, 4 * g + 2)
        n = int(round(math.exp(lo + u0 * (hi - lo))))
        n = min(max(n, nmin), nmax)
        if g % 2 == 0:
            specs.append(BatchSpec("er", n, er_deg[0] + u1 * (er_deg[1] - er_deg[0]), gseed))
        else:
            specs.append(BatchSpec("rmat", n, rmat_ef[0] + u1 * (rmat_ef[1] - rmat_ef[0]), gseed))
    return specs


def make_from_spec(s: BatchSpec) -> Graph:
    if s.kind == "er":
        return er(s.n, s.param, s.seed)
    if s.kind == "rmat":
        scale = max(1, int(math.ceil(math.log2(s.n))))
        return rmat(scale, s.param, s.seed, n=s.n)
    if s.kind == "grid":
        side = max(1, int(round(math.sqrt(s.n))))
        return grid5(side, max(1, s.n // side))
    raise ValueError(s.kind)


@dataclass
class Batch:
    """Graphs packed back to back.  Graph g's vertices occupy [vtx_off[g], vtx_off[g+1]) of the
    color array, its own (n_g+1)-entry local rowptr starts at rowptr[vtx_off[g] + g], and its local
    column ids start at colidx[edge_off[g]]."""

    G: int
    vtx_off: np.ndarray  # int64[G+1]
    edge_off: np.ndarray  # int64[G+1]
    rowptr: np.ndarray  # int32[vtx_off[G] + G]
    colidx: np.ndarray  # int32[edge_off[G]]

    def graph(self, g: int) -> Graph:
        v0, v1 = int(self.vtx_off[g]), int(self.vtx_off[g + 1])
        e0, e1 = int(self.edge_off[g]), int(self.edge_off[g + 1])
        rp = self.rowptr[v0 + g: v1 + g + 1]
        return Graph(v1 - v0, rp, self.colidx[e0:e1], name=f"batch[{g}]")


def pack(graphs: list[Graph]) -> Batch:
    G = len(graphs)
    vtx_off = np.zeros(G + 1, dtype=np.int64)
    edge_off = np.zeros(G + 1, dtype=np.int64)
    for g, gr in enumerate(graphs):
        vtx_off[g + 1] = vtx_off[g] + gr.n
        edge_off[g + 1] = edge_off[g] + gr.nnz
    rowptr = np.empty(int(vtx_off[G]) + G, dtype=np.int32)
    colidx = np.empty(int(edge_off[G]), dtype=np.int32)
    for g, gr in enumerate(graphs):
        v0 = int(vtx_off[g])
        rowptr[v0 + g: v0 + g + gr.n + 1] = gr.rowptr
        colidx[int(edge_off[g]): int(edge_off[g + 1])] = gr.colidx[: gr.nnz]
    return Batch(G, vtx_off, edge_off, rowptr, colidx)


def batch_mix(G: int, seed: int, **kw) -> Batch:
    """The batch of batch_specs(G, seed, ...), generated in parallel in C (same graphs as
    make_from_spec graph by graph)."""
    specs = batch_specs(G, seed, **kw)
    if any(s.kind not in ("er", "rmat") for s in specs):
        return pack([make_from_spec(s) for s in specs])
    kind = np.array([0 if s.kind == "er" else 1 for s in specs], np.int32)
    n = np.array([s.n for s in specs], np.int32)
    param = np.array([s.param for s in specs], np.float64)
    seeds = np.array([s.seed for s in specs], np.uint64)
    M = np.array([_round_half_up(s.n * s.param / 2) if s.kind == "er" else _round_half_up(s.n * s.param)
                  for s in specs], np.int64)
    M[n < 2] = 0
    vtx_off = np.zeros(G + 1, np.int64)
    vtx_off[1:] = np.cumsum(n)
    cap_off = np.zeros(G + 1, np.int64)
    cap_off[1:] = np.cumsum(2 * M)
    rowptr = np.empty(int(vtx_off[-1]) + G, np.int32)
    colidx = np.empty(max(int(cap_off[-1]), 1), np.int32)
    nnz = np.zeros(G, np.int64)
    if _L().gg_batch(G, kind.ctypes.data, n.ctypes.data, param.ctypes.data, seeds.ctypes.data, 0.57, 0.19, 0.19,
                     PERM_STREAM_OFFSET, vtx_off.ctypes.data, cap_off.ctypes.data, rowptr.ctypes.data,
                     colidx.ctypes.data, nnz.ctypes.data) != 0:
        raise MemoryError("gg_batch")
    edge_off = np.zeros(G + 1, np.int64)
    edge_off[1:] = np.cumsum(nnz)
    _L().gg_batch_pack(G, cap_off.ctypes.data, edge_off.ctypes.data, colidx.ctypes.data)
    return Batch(G, vtx_off, edge_off, rowptr, colidx[: int(edge_off[-1])])


# ---------------------------------------------------------------------------------------------
# named workloads with an on-disk cache

def cache_dir() -> str:
    d = os.environ.get("GC_GRAPH_CACHE", os.path.join("/tmp", "gc_graph_cache"))
    os.makedirs(d, exist_ok=True)
    return d


def cached(key: str, make) -> Graph:
    path = os.path.join(cache_dir(), key + ".npz")
    if os.path.exists(path):
        try:
            z = np.load(path)
            return Graph(int(z["n"]), z["rowptr"], z["colidx"], name=key)
        except Exception:
            pass
    g = make()
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, n=np.int64(g.n), rowptr=g.rowptr, colidx=g.colidx)
    os.replace(tmp, path)
    g.name = key
    return g


WORKLOADS = {
    # Erdos-Renyi n=10,000, average degree 16, edge seed 1 (colored with hash seed 7)
    "er10k": lambda: er(10_000, 16, 1),
    # R-MAT scale 22, edge factor 16, a=.57 b=.19 c=.19, seed 2, permuted ids
    "rmat22": lambda: rmat(22, 16, 2),
    # 3-D 27-point stencil 256^3, natural ids
    "stencil256": lambda: stencil27(256),
}


def workload(name: str) -> Graph:
    """A named workload; small variants such as 'rmat16' or 'stencil32' are generated on demand."""
    if name in WORKLOADS:
        return cached(name, WORKLOADS[name])
    if name.startswith("rmat"):
        s = int(name[4:])
        return cached(name, lambda: rmat(s, 16, 2))
    if name.startswith("stencil"):
        L = int(name[7:])
        return cached(name, lambda: stencil27(L))
    raise KeyError(name)
