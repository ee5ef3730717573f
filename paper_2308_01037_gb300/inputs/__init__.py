"""Seeded synthetic input graphs shared by the CUDA path's tests, the oracle's
tests and the benchmark.

This module draws graphs only; it contains none of the Monte Carlo method's
arithmetic.  Every undirected generator returns a :class:`Graph` holding a
symmetric, loop-free, duplicate-free CSR adjacency structure (``row_ptr``
int64 of length n+1, ``col_idx`` int32, rows sorted) -- the matrix class of the
paper's Section 2.1; the ``directed_*`` generators return a general
(non-symmetric) A in the same layout, and ``bipartite_symmetrization`` turns
one into the symmetric B of the paper's Section 4.  The C implementation lives in ``graphgen.c`` and is compiled on
first use with the host C compiler.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(os.path.dirname(_HERE), "_build")
_SO = os.path.join(_BUILD, "libgraphgen.so")
_SRC = os.path.join(_HERE, "graphgen.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles ``graphgen.c`` into ``_build/libgraphgen.so`` and returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
            lib.gg_rmat.argtypes = [i32, i32, dbl, dbl, dbl, u64, i32]
            lib.gg_ba.argtypes = [i64, i32, u64]
            lib.gg_er.argtypes = [i64, dbl, u64]
            lib.gg_config_powerlaw.argtypes = [i64, dbl, dbl, u64]
            lib.gg_smallworld.argtypes = [i64, i32, dbl, u64]
            lib.gg_from_edges.argtypes = [i64, i64, P, P]
            for f in ("gg_rmat", "gg_ba", "gg_er", "gg_config_powerlaw", "gg_smallworld", "gg_from_edges"):
                getattr(lib, f).restype = P
            lib.gg_n.argtypes = [P]
            lib.gg_n.restype = i64
            lib.gg_nnz.argtypes = [P]
            lib.gg_nnz.restype = i64
            lib.gg_copy.argtypes = [P, P, P]
            lib.gg_copy.restype = None
            lib.gg_free.argtypes = [P]
            lib.gg_free.restype = None
            _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected graph in CSR form (int64 row pointers, int32 sorted columns)."""

    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def degree(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def dense(self) -> np.ndarray:
        """Dense float64 adjacency matrix (small graphs only)."""
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), self.degree)
        a[rows, self.col_idx] = 1.0
        return a


def _take(ptr, name: str) -> Graph:
    lib = _load()
    if not ptr:
        raise MemoryError(f"graph generator {name} failed")
    try:
        n = lib.gg_n(ptr)
        nnz = lib.gg_nnz(ptr)
        rp = np.empty(n + 1, dtype=np.int64)
        ci = np.empty(max(nnz, 1), dtype=np.int32)
        lib.gg_copy(ptr, rp.ctypes.data, ci.ctypes.data)
    finally:
        lib.gg_free(ptr)
    return Graph(int(n), rp, ci[:nnz].copy(), name)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, permute: bool = True) -> Graph:
    """Graph500-style R-MAT graph on 2**scale nodes, symmetrised and deduplicated."""
    return _take(_load().gg_rmat(scale, edge_factor, a, b, c, seed, int(permute)),
                 f"rmat{scale}_ef{edge_factor}_s{seed}")


def barabasi_albert(n: int, m: int, seed: int = 0) -> Graph:
    return _take(_load().gg_ba(n, m, seed), f"ba_n{n}_m{m}_s{seed}")


def erdos_renyi(n: int, mean_degree: float, seed: int = 0) -> Graph:
    return _take(_load().gg_er(n, mean_degree, seed), f"er_n{n}_d{mean_degree:g}_s{seed}")


def config_powerlaw(n: int, exponent: float = 2.5, mean_degree: float = 20.0, seed: int = 2) -> Graph:
    return _take(_load().gg_config_powerlaw(n, exponent, mean_degree, seed),
                 f"cm_n{n}_g{exponent:g}_d{mean_degree:g}_s{seed}")


def smallworld(n: int, k: int = 10, p: float = 0.1, seed: int = 0) -> Graph:
    return _take(_load().gg_smallworld(n, k, p, seed), f"ws_n{n}_k{k}_s{seed}")


def from_edges(n: int, edges, name: str = "") -> Graph:
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    src = np.ascontiguousarray(e[:, 0])
    dst = np.ascontiguousarray(e[:, 1])
    return _take(_load().gg_from_edges(n, len(e), src.ctypes.data, dst.ctypes.data), name or f"edges_n{n}")


def complete(n: int) -> Graph:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"K{n}")


def path(n: int) -> Graph:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], f"P{n}")


def cycle(n: int) -> Graph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], f"C{n}")


def star(n: int) -> Graph:
    """Star on n nodes: node 0 is the centre."""
    return from_edges(n, [(0, i) for i in range(1, n)], f"S{n}")


def add_isolated(g: Graph, k: int) -> Graph:
    """Returns g with k isolated nodes appended (ids n..n+k-1)."""
    rp = np.concatenate([g.row_ptr, np.full(k, g.row_ptr[-1], dtype=np.int64)])
    return Graph(g.n + k, rp, g.col_idx.copy(), g.name + f"+{k}iso")


def symmetric_weights(g: Graph, seed: int = 0, signed: bool = False, low: float = 0.25,
                      high: float = 2.0) -> np.ndarray:
    """float32 edge values with a_ij = a_ji, |a| uniform in [low, high), random sign when ``signed``."""
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), g.degree)
    cols = g.col_idx.astype(np.int64)
    lo = np.minimum(rows, cols)
    hi = np.maximum(rows, cols)
    key = lo * g.n + hi
    uniq, inv = np.unique(key, return_inverse=True)
    mag = rng.uniform(low, high, size=len(uniq))
    sgn = np.where(rng.random(len(uniq)) < 0.5, -1.0, 1.0) if signed else np.ones(len(uniq))
    return (mag * sgn)[inv].astype(np.float32)


# ---------------------------------------------------------------- directed graphs
def directed_from_edges(n: int, src, dst, name: str = "") -> Graph:
    """Directed CSR (row i lists the heads j of the arcs i -> j, sorted, no
    duplicates; loops kept): a general, non-symmetric A."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    key = np.unique(src * n + dst)
    rows, cols = key // n, key % n
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    return Graph(n, np.cumsum(rp), cols.astype(np.int32), name or f"digraph_n{n}")


def directed_erdos_renyi(n: int, mean_out_degree: float, seed: int, loops: bool = False) -> Graph:
    """Directed G(n, p), p = mean_out_degree / n: arcs drawn independently."""
    rng = np.random.default_rng(seed)
    m = rng.binomial(n * n, min(1.0, mean_out_degree / n))
    key = np.unique(rng.integers(0, n * n, size=m, dtype=np.int64))
    src, dst = key // n, key % n
    if not loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    return directed_from_edges(n, src, dst, f"dER_n{n}_k{mean_out_degree:g}_s{seed}")


def directed_cycle(n: int) -> Graph:
    """Directed cycle i -> i + 1 (mod n): the permutation matrix P with P^n = I."""
    i = np.arange(n)
    return directed_from_edges(n, i, (i + 1) % n, f"dC{n}")


def bipartite_symmetrization(g: Graph, values=None):
    """B = [0 A; A^T 0] of a directed graph (Section 4, Eq. digraph_sym): node
    i keeps the out-arcs of i, node n + i its in-arcs.  Returns the symmetric
    graph on 2n nodes and, if ``values`` is given, B's values in CSR order."""
    n = g.n
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.row_ptr))
    cols = g.col_idx.astype(np.int64)
    src = np.concatenate([rows, n + cols])
    dst = np.concatenate([n + cols, rows])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    rp = np.zeros(2 * n + 1, dtype=np.int64)
    np.add.at(rp, src + 1, 1)
    b = Graph(2 * n, np.cumsum(rp), dst.astype(np.int32), f"B({g.name})")
    if values is None:
        return b
    w = np.concatenate([np.asarray(values, np.float32)] * 2)[order]
    return b, w
