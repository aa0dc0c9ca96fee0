"""CPU oracle for the Wedge hot path (TEST INFRASTRUCTURE ONLY).

A plain restatement, in C (``oracle.c``) behind this ctypes wrapper, of what
the paper's method computes: BFS, connected components (HCC), SSSP
(Bellman-Ford and Dijkstra), FP64 PageRank, the Wedge Frontier by definition
and through the edge index, the frontier fullness, and a whole Wedge run with
its per-iteration trace.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the engine never does,
and the two share no code.

Every function takes a graph as any object with ``V``, ``offsets`` (uint32,
V+1), ``src`` (uint32, E) and, for SSSP, ``w`` (uint32, E) in CSC order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lib = None

INF = 0xFFFFFFFF
BFS, CC, SSSP = 0, 1, 2
POLICY_THRESHOLD, POLICY_ALWAYS_DENSE, POLICY_ALWAYS_SPARSE = 0, 1, 2
APPS = {"bfs": BFS, "cc": CC, "sssp": SSSP}


def build(force: bool = False) -> str:
    """Compile oracle.c (plain C11, -O2) into _oracle.so.  Everything is
    single-threaded except the *_omp timing variants, which share their
    destination loop among OpenMP threads when gcc has -fopenmp."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:5] + ["-fopenmp"] + base[5:], capture_output=True)
    if r.returncode != 0:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u32, u64, i32, dbl, p = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        sig = {
            "or_csc_to_csr": (None, [u32, u64, p, p, p, p, p]),
            "or_outdeg": (None, [u32, u64, p, p]),
            "or_bfs_push": (None, [u32, p, p, u32, p]),
            "or_cc_union_find": (None, [u32, p, p, p]),
            "or_sssp_dijkstra": (None, [u32, u64, p, p, p, p, u32, p]),
            "or_sssp_push": (None, [u32, p, p, p, p, u32, p]),
            "or_pr_pull": (None, [u32, p, p, p, dbl, u32, p]),
            "or_pr_push": (None, [u32, p, p, dbl, u32, p]),
            "or_in_sums": (None, [u32, p, p, p, p]),
            "or_wedge_groups_scan": (u64, [u64, p, p, u64, p]),
            "or_edge_index": (u64, [u32, u64, p, p, u64, p, p]),
            "or_wedge_groups_index": (u64, [u32, p, p, p, u64, p]),
            "or_fullness": (u64, [u32, p, p]),
            "or_wedge_run": (u64, [i32, u32, u64, p, p, p, u32, i32, u32, u64, u64, p, p, u64]),
            "or_omp_threads": (i32, []),
            "or_dense_pull_omp": (u64, [i32, u32, p, p, p, u32, p]),
            "or_pr_pull_omp": (None, [u32, p, p, p, dbl, u32, p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _P(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def _graph(g):
    return int(g.V), _c(g.offsets, np.uint32), _c(g.src, np.uint32)


def outdeg(g) -> np.ndarray:
    V, off, src = _graph(g)
    out = np.empty(V, dtype=np.uint32)
    _load().or_outdeg(V, src.size, _P(src), _P(out))
    return out


def csr(g):
    """Out-edge view: (csr_off[V+1] u64, csr_dst[E] u32, csr_pos[E] u64)."""
    V, off, src = _graph(g)
    E = src.size
    co = np.empty(V + 1, dtype=np.uint64)
    cd = np.empty(E, dtype=np.uint32)
    cp = np.empty(E, dtype=np.uint64)
    _load().or_csc_to_csr(V, E, _P(off), _P(src), _P(co), _P(cd), _P(cp))
    return co, cd, cp


def bfs_push(g, root: int) -> np.ndarray:
    co, cd, _ = csr(g)
    lvl = np.empty(int(g.V), dtype=np.uint32)
    _load().or_bfs_push(int(g.V), _P(co), _P(cd), root, _P(lvl))
    return lvl


def cc_union_find(g) -> np.ndarray:
    V, off, src = _graph(g)
    lab = np.empty(V, dtype=np.uint32)
    _load().or_cc_union_find(V, _P(off), _P(src), _P(lab))
    return lab


def sssp_dijkstra(g, root: int) -> np.ndarray:
    co, cd, cp = csr(g)
    w = _c(g.w, np.uint32)
    dist = np.empty(int(g.V), dtype=np.uint32)
    _load().or_sssp_dijkstra(int(g.V), w.size, _P(co), _P(cd), _P(cp), _P(w), root, _P(dist))
    return dist


def sssp_push(g, root: int) -> np.ndarray:
    co, cd, cp = csr(g)
    w = _c(g.w, np.uint32)
    dist = np.empty(int(g.V), dtype=np.uint32)
    _load().or_sssp_push(int(g.V), _P(co), _P(cd), _P(cp), _P(w), root, _P(dist))
    return dist


def pr_pull(g, damping: float = 0.85, iters: int = 20) -> np.ndarray:
    V, off, src = _graph(g)
    od = outdeg(g)
    pr = np.empty(V, dtype=np.float64)
    _load().or_pr_pull(V, _P(off), _P(src), _P(od), damping, iters, _P(pr))
    return pr


def in_sums(g, x) -> np.ndarray:
    """FP64 in-edge sums of the per-vertex values x (PageRank's in-edge pass
    when x = pr/outdeg)."""
    _, off, src = _graph(g)
    xx = _c(np.asarray(x, dtype=np.float64), np.float64)
    out = np.empty(int(g.V), dtype=np.float64)
    _load().or_in_sums(int(g.V), _P(off), _P(src), _P(xx), _P(out))
    return out


def pr_push(g, damping: float = 0.85, iters: int = 20) -> np.ndarray:
    co, cd, _ = csr(g)
    pr = np.empty(int(g.V), dtype=np.float64)
    _load().or_pr_push(int(g.V), _P(co), _P(cd), damping, iters, _P(pr))
    return pr


def _front_bytes(V: int, frontier) -> np.ndarray:
    f = np.asarray(frontier)
    if f.dtype == bool or (f.size == V and f.dtype == np.uint8):
        out = f.astype(np.uint8)
        if out.size != V:
            raise ValueError("frontier mask must have V entries")
        return np.ascontiguousarray(out)
    out = np.zeros(V, dtype=np.uint8)
    out[f.astype(np.int64)] = 1
    return out


def wedge_groups_scan(g, frontier, group: int = 32) -> np.ndarray:
    """Wedge Frontier by definition: sorted groups of `group` consecutive CSC
    positions holding an edge whose source is in `frontier` (vertex ids or a
    V-long boolean mask)."""
    V, off, src = _graph(g)
    fb = _front_bytes(V, frontier)
    out = np.empty(max(src.size, 1), dtype=np.uint64)
    n = _load().or_wedge_groups_scan(src.size, _P(src), _P(fb), group, _P(out))
    return out[:n].copy()


def edge_index(g, group: int = 32):
    """(eidx_off[V+1], eidx[]) with sorted, de-duplicated group ids per source."""
    V, off, src = _graph(g)
    eo = np.empty(V + 1, dtype=np.uint64)
    ei = np.empty(max(src.size, 1), dtype=np.uint64)
    n = _load().or_edge_index(V, src.size, _P(off), _P(src), group, _P(eo), _P(ei))
    return eo, ei[:n].copy()


def wedge_groups_index(g, frontier, group: int = 32, index=None) -> np.ndarray:
    """Wedge Frontier through the edge index (the paper's transformation)."""
    V, off, src = _graph(g)
    eo, ei = index if index is not None else edge_index(g, group)
    eo = _c(eo, np.uint64)
    ei = _c(ei, np.uint64)
    fb = _front_bytes(V, frontier)
    ngroups = (src.size + group - 1) // group
    out = np.empty(max(ngroups, 1), dtype=np.uint64)
    n = _load().or_wedge_groups_index(V, _P(eo), _P(ei), _P(fb), ngroups, _P(out))
    return out[:n].copy()


def fullness(g, frontier) -> int:
    V, _, _ = _graph(g)
    od = outdeg(g)
    fb = _front_bytes(V, frontier)
    return int(_load().or_fullness(V, _P(od), _P(fb)))


def wedge_run(app, g, root: int = 0, policy: int = POLICY_THRESHOLD, tau_bp: int = 100,
              group: int = 32, max_iters: int = 1 << 20, trace_cap: int = 1 << 16):
    """Whole Wedge run.  Returns (values uint32[V], trace uint64[iters, 5]) with
    trace columns |F_t|, fullness(F_t), mode (1 = Wedge Frontier), groups
    pulled, edges pulled."""
    a = APPS[app] if isinstance(app, str) else int(app)
    V, off, src = _graph(g)
    if a == SSSP:
        w = _c(g.w, np.uint32)
    else:
        w = np.zeros(0, dtype=np.uint32)
    vals = np.empty(V, dtype=np.uint32)
    trace = np.zeros(5 * trace_cap, dtype=np.uint64)
    it = _load().or_wedge_run(a, V, src.size, _P(off), _P(src), _P(w), root, policy, tau_bp,
                              group, max_iters, _P(vals), _P(trace), trace_cap)
    return vals, trace[: 5 * min(it, trace_cap)].reshape(-1, 5)


def bfs_pull(g, root: int) -> np.ndarray:
    return wedge_run("bfs", g, root, POLICY_ALWAYS_DENSE)[0]


def cc_pull(g) -> np.ndarray:
    return wedge_run("cc", g, 0, POLICY_ALWAYS_DENSE)[0]


def sssp_pull(g, root: int) -> np.ndarray:
    return wedge_run("sssp", g, root, POLICY_ALWAYS_DENSE)[0]


# ---- all-cores timing variants (the CPU baseline's multi-threaded leg) ----

def omp_threads() -> int:
    """Threads the *_omp variants use (1 without OpenMP)."""
    return int(_load().or_omp_threads())


def dense_pull_omp(app, g, root: int = 0) -> tuple[np.ndarray, int]:
    """BFS/CC/SSSP by dense pulls, destinations shared among threads:
    (values, pulls); the values equal the single-threaded pull's."""
    a = APPS[app] if isinstance(app, str) else int(app)
    V, off, src = _graph(g)
    w = _c(g.w, np.uint32) if a == SSSP else np.zeros(1, dtype=np.uint32)
    vals = np.empty(V, dtype=np.uint32)
    it = _load().or_dense_pull_omp(a, V, _P(off), _P(src), _P(w), root, _P(vals))
    return vals, int(it)


def pr_pull_omp(g, damping: float = 0.85, iters: int = 20) -> np.ndarray:
    V, off, src = _graph(g)
    od = outdeg(g)
    pr = np.empty(V, dtype=np.float64)
    _load().or_pr_pull_omp(V, _P(off), _P(src), _P(od), damping, iters, _P(pr))
    return pr
