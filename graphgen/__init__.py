"""Seeded synthetic graph inputs shared by the oracle and the CUDA engine.

Holds none of the method's arithmetic: it only produces graphs in the
destination-sorted CSC layout (offsets[V+1], src[E], optional w[E]), SSSP
weights and roots.  The heavy loops live in ``graphgen.c`` (compiled here on
first use with gcc; OpenMP when available) and every draw is addressed by a
counter, so results do not depend on the thread count.

Seed table (fixed by the workload recipes): graph = 1, weights = 2,
roots = 3, grid rewiring = 4.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "_graphgen.so")
_lib = None

SEED_GRAPH, SEED_WEIGHTS, SEED_ROOTS, SEED_REWIRE = 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile graphgen.c into _graphgen.so (OpenMP if the compiler has it)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        p = ctypes.c_void_p
        lib.gg_rand.restype = u64
        lib.gg_rand.argtypes = [u64, u64]
        lib.gg_weight.restype = u32
        lib.gg_weight.argtypes = [u32, u32, u32, u32]
        lib.gg_rmat_keys.restype = None
        lib.gg_rmat_keys.argtypes = [i32, u64, u32, u32, u32, u64, p]
        lib.gg_grid_keys.restype = u64
        lib.gg_grid_keys.argtypes = [u32, u64, u64, p]
        lib.gg_add_reverse.restype = u64
        lib.gg_add_reverse.argtypes = [p, u64]
        lib.gg_sort_unique.restype = u64
        lib.gg_sort_unique.argtypes = [p, p, u64, i32]
        lib.gg_keys_to_csc.restype = None
        lib.gg_keys_to_csc.argtypes = [p, u64, u32, p, p]
        lib.gg_csc_weights.restype = None
        lib.gg_csc_weights.argtypes = [p, p, u32, u32, u32, i32, p]
        lib.gg_outdeg.restype = None
        lib.gg_outdeg.argtypes = [p, u64, u32, p]
        lib.gg_roots.restype = None
        lib.gg_roots.argtypes = [p, u32, u64, u32, p]
        lib.gg_num_threads.restype = i32
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Graph:
    """A directed graph in CSC form: the in-edges of v are src[offsets[v]:offsets[v+1]],
    sorted by source id.  ``w`` (same order as ``src``) is None when unweighted."""

    V: int
    offsets: np.ndarray
    src: np.ndarray
    w: np.ndarray | None = None
    name: str = "graph"
    undirected: bool = False
    params: dict = field(default_factory=dict)

    @property
    def E(self) -> int:
        return int(self.src.shape[0])

    def outdeg(self) -> np.ndarray:
        out = np.empty(self.V, dtype=np.uint32)
        _load().gg_outdeg(_ptr(self.src), self.E, self.V, _ptr(out))
        return out

    def indeg(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64)).astype(np.uint32)

    def dst(self) -> np.ndarray:
        """Destination of every CSC position (an expanded copy, for tests)."""
        return np.repeat(np.arange(self.V, dtype=np.uint32), self.indeg().astype(np.int64))

    def with_weights(self, wmax: int, seed: int = SEED_WEIGHTS) -> "Graph":
        w = np.empty(self.E, dtype=np.uint32)
        _load().gg_csc_weights(_ptr(self.offsets), _ptr(self.src), self.V, seed, wmax,
                               1 if self.undirected else 0, _ptr(w))
        params = dict(self.params, wmax=wmax, wseed=seed)
        return Graph(self.V, self.offsets, self.src, w, self.name, self.undirected, params)


def _vbits(V: int) -> int:
    return max(1, int(V - 1).bit_length())


def _from_keys(keys: np.ndarray, n: int, V: int, name: str, undirected: bool, params: dict) -> Graph:
    lib = _load()
    tmp = np.empty(n, dtype=np.uint64)
    E = lib.gg_sort_unique(_ptr(keys), _ptr(tmp), n, _vbits(V))
    del tmp
    if E >= 2**32 - 1:
        raise ValueError("graph has too many edges for 32-bit positions")
    offsets = np.empty(V + 1, dtype=np.uint32)
    src = np.empty(E, dtype=np.uint32)
    lib.gg_keys_to_csc(_ptr(keys), E, V, _ptr(offsets), _ptr(src))
    return Graph(V, offsets, src, None, name, undirected, params)


def _thresholds(a: float, b: float, c: float):
    def q(x):
        return min(int(x * 2**32), 2**32 - 1)
    return q(a), q(a + b), q(a + b + c)


def rmat(scale: int, ef: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = SEED_GRAPH) -> Graph:
    """R-MAT graph with 2^scale vertices from ef * 2^scale samples (directed)."""
    V = 1 << scale
    m = ef << scale
    keys = np.empty(m, dtype=np.uint64)
    ta, tab, tabc = _thresholds(a, b, c)
    _load().gg_rmat_keys(scale, m, ta, tab, tabc, seed, _ptr(keys))
    return _from_keys(keys, m, V, f"rmat-s{scale}-ef{ef}", False,
                      dict(kind="rmat", scale=scale, ef=ef, a=a, b=b, c=c, seed=seed))


def grid(n: int, p: float = 0.01, seed: int = SEED_REWIRE) -> Graph:
    """n x n 4-neighbour grid, each undirected edge rewired with probability p."""
    V = n * n
    keys = np.empty(4 * V, dtype=np.uint64)
    thresh = 0 if p <= 0 else min(int(p * 2**64), 2**64 - 1)
    cnt = _load().gg_grid_keys(n, thresh, seed, _ptr(keys))
    return _from_keys(keys, cnt, V, f"grid-{n}x{n}-p{p:g}", True,
                      dict(kind="grid", n=n, p=p, seed=seed))


def symmetrize(g: Graph) -> Graph:
    """E union E^T, deduplicated (used for connected components)."""
    dst = g.dst().astype(np.uint64)
    n = g.E
    keys = np.empty(2 * n, dtype=np.uint64)
    keys[:n] = (dst << np.uint64(32)) | g.src.astype(np.uint64)
    _load().gg_add_reverse(_ptr(keys), n)
    out = _from_keys(keys, 2 * n, g.V, g.name + "-sym", True, dict(g.params, symmetrized=True))
    return out


def from_edges(V: int, src, dst, w=None, undirected: bool = False, name: str = "edges") -> Graph:
    """Graph from explicit edge lists (small test graphs).  Self-loops and
    duplicates are dropped; if w is given it is carried along (first copy of a
    duplicated edge wins)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= V or dst.max() >= V):
        raise ValueError("vertex id out of range")
    keep = src != dst
    src, dst = src[keep], dst[keep]
    order = np.lexsort((src, dst))
    src, dst = src[order], dst[order]
    if src.size:
        uniq = np.ones(src.size, dtype=bool)
        uniq[1:] = (src[1:] != src[:-1]) | (dst[1:] != dst[:-1])
    else:
        uniq = np.ones(0, dtype=bool)
    src, dst = src[uniq], dst[uniq]
    offsets = np.zeros(V + 1, dtype=np.uint32)
    np.add.at(offsets, dst + 1, 1)
    offsets = np.cumsum(offsets, dtype=np.uint64).astype(np.uint32)
    ww = None
    if w is not None:
        ww = np.asarray(w, dtype=np.uint32)[keep][order][uniq]
    return Graph(V, offsets, src.astype(np.uint32), ww, name, undirected, dict(kind="edges"))


def random_graph(V: int, m: int, seed: int, undirected: bool = False) -> Graph:
    """Uniform random directed graph with m samples (small test graphs)."""
    lib = _load()
    r = np.array([lib.gg_rand(seed, i) for i in range(2 * m)], dtype=np.uint64)
    s = (r[0::2] % np.uint64(max(V, 1))).astype(np.int64)
    d = (r[1::2] % np.uint64(max(V, 1))).astype(np.int64)
    if undirected:
        s, d = np.concatenate([s, d]), np.concatenate([d, s])
    return from_edges(V, s, d, undirected=undirected, name=f"random-{V}-{m}-{seed}")


def block_diagonal(graphs) -> tuple[Graph, np.ndarray]:
    """Concatenates graphs into one CSC with disjoint vertex ranges (graph i's
    vertex v becomes base[i] + v).  Returns (graph, base offsets)."""
    base = np.zeros(len(graphs) + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        base[i + 1] = base[i] + g.V
    V = int(base[-1])
    E = sum(g.E for g in graphs)
    if E >= 2**32 - 1 or V >= 2**32:
        raise ValueError("batch too large for 32-bit ids")
    offsets = np.empty(V + 1, dtype=np.uint32)
    src = np.empty(E, dtype=np.uint32)
    w = np.empty(E, dtype=np.uint32) if all(g.w is not None for g in graphs) else None
    e0 = 0
    for i, g in enumerate(graphs):
        offsets[base[i]:base[i + 1]] = g.offsets[:-1].astype(np.int64) + e0
        src[e0:e0 + g.E] = g.src.astype(np.int64) + base[i]
        if w is not None:
            w[e0:e0 + g.E] = g.w
        e0 += g.E
    offsets[V] = E
    return Graph(V, offsets, src, w, f"batch-{len(graphs)}", False, dict(kind="block-diagonal")), base[:-1]


def roots(g: Graph, count: int, seed: int = SEED_ROOTS) -> np.ndarray:
    """`count` roots uniform (with replacement) over vertices with outdeg > 0."""
    od = g.outdeg()
    out = np.empty(count, dtype=np.uint32)
    _load().gg_roots(_ptr(od), g.V, seed, count, _ptr(out))
    return out


def weight(u: int, v: int, seed: int, wmax: int) -> int:
    return int(_load().gg_weight(u, v, seed, wmax))


def rand(seed: int, n: int) -> int:
    return int(_load().gg_rand(seed, n))


def num_threads() -> int:
    return int(_load().gg_num_threads())
