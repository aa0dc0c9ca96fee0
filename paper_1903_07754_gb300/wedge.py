"""Thin ctypes binding over libwedge.so (include/wedge.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Functions carry the C names; tensors are passed by data
pointer and the stream is torch's current stream unless one is given.  The
binding raises if the library cannot be loaded: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwedge.so")

BFS, CC, SSSP, PR = 0, 1, 2, 3
APP_IDS = {"bfs": BFS, "cc": CC, "sssp": SSSP, "pr": PR}
SWITCH_THRESHOLD, SWITCH_LEARNED, SWITCH_ALWAYS_DENSE, SWITCH_ALWAYS_SPARSE = 0, 1, 2, 3
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA", 4: "TIMEOUT", 5: "NOT_SUPPORTED",
          6: "MAX_ITERS"}
INF = 0xFFFFFFFF


class WedgeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"wedge {STATUS.get(status, status)}: {msg}")
        self.status = status


class wedge_opts(ctypes.Structure):
    _fields_ = [("tau_bp", ctypes.c_uint32), ("log2_coarsen", ctypes.c_uint32),
                ("switch_mode", ctypes.c_uint32), ("max_iters", ctypes.c_uint32),
                ("trace", ctypes.c_uint32), ("synchronous", ctypes.c_uint32),
                ("sparse_push", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 1)]


class wedge_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_uint32), ("sparse_iters", ctypes.c_uint32),
                ("edges_pulled", ctypes.c_uint64), ("chunks_listed", ctypes.c_uint64),
                ("device_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class wedge_iter_record(ctypes.Structure):
    _fields_ = [("fullness", ctypes.c_uint64), ("nfront", ctypes.c_uint32), ("mode", ctypes.c_uint32),
                ("log2_coarsen", ctypes.c_uint32), ("nchunks", ctypes.c_uint32), ("rowsum", ctypes.c_uint32),
                ("npieces", ctypes.c_uint32), ("t_pull_ns", ctypes.c_uint64), ("t_xform_ns", ctypes.c_uint64)]


class wedge_tuning(ctypes.Structure):
    _fields_ = [("dense_loader", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("edge_index", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 5)]


class wedge_graph_info(ctypes.Structure):
    _fields_ = [("V", ctypes.c_uint32), ("nz_dst", ctypes.c_uint32), ("E", ctypes.c_uint64),
                ("nchunks", ctypes.c_uint64), ("eidx_len", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("device", ctypes.c_int), ("eidx_bytes", ctypes.c_uint64), ("eidx_z_bytes", ctypes.c_uint64),
                ("eidx_z_blocks", ctypes.c_uint64), ("eidx_z_words", ctypes.c_uint64)]


EXPORTS = [
    "wedge_default_opts", "wedge_graph_create", "wedge_graph_destroy", "wedge_graph_get_info",
    "wedge_graph_copy_edge_index", "wedge_frontier_transform", "wedge_pull_iterate", "wedge_run_bfs",
    "wedge_run_cc", "wedge_run_sssp", "wedge_run_pr", "wedge_get_trace", "wedge_kernel_launches",
    "wedge_last_error", "wedge_version", "wedge_graph_set_tuning", "wedge_graph_get_tuning",
    "wedge_frontier_transform_noalloc", "wedge_mlp_forward", "wedge_mlp_forward_bf16", "wedge_mlp_loss_grad",
    "wedge_mlp_adam", "wedge_set_cost_model", "wedge_trace_candidates", "wedge_run_bfs_batch",
    "wedge_pr_pull", "wedge_trim_memory", "wedge_selftest_timeout", "wedge_run_sssp_batch",
    "wedge_frontier_transform_profile", "wedge_graph_copy_edge_index_z", "wedge_set_learned_band",
    "wedge_csc_relabel_by_degree", "wedge_permute_rows", "wedge_cc_labels_to_original", "wedge_run_bfs_batch_u8",
    "wedge_pr_order", "wedge_pr_pull_ordered",
]
MLP_FEATURES, MLP_PARAMS, MLP_CANDIDATES = 12, 5057, 6

_lib = None


def load(path: str = LIB_PATH):
    """Loads libwedge.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(path)
    P, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    st = ctypes.c_int
    sig = {
        "wedge_default_opts": (None, [i32, ctypes.POINTER(wedge_opts)]),
        "wedge_graph_create": (st, [u32, u64, P, P, P, P, P, u32, P, ctypes.POINTER(P)]),
        "wedge_graph_destroy": (st, [P]),
        "wedge_graph_get_info": (st, [P, ctypes.POINTER(wedge_graph_info)]),
        "wedge_graph_copy_edge_index": (st, [P, P, P, P]),
        "wedge_frontier_transform": (st, [P, P, u32, P, P, P]),
        "wedge_frontier_transform_noalloc": (st, [u32, u64, P, P, P, u32, P, P, P]),
        "wedge_frontier_transform_profile": (st, [P, P, u32, u32, P, P, P, u32, ctypes.POINTER(u32), P]),
        "wedge_graph_copy_edge_index_z": (st, [P, P, P, P, P]),
        "wedge_set_learned_band": (st, [P, ctypes.c_float, ctypes.c_float]),
        "wedge_pull_iterate": (st, [P, i32, P, u32, P, P, P, u32, P, P, P, P]),
        "wedge_run_bfs": (st, [P, u32, P, ctypes.POINTER(wedge_opts), ctypes.POINTER(wedge_stats), P]),
        "wedge_run_cc": (st, [P, P, ctypes.POINTER(wedge_opts), ctypes.POINTER(wedge_stats), P]),
        "wedge_run_sssp": (st, [P, u32, P, ctypes.POINTER(wedge_opts), ctypes.POINTER(wedge_stats), P]),
        "wedge_pr_pull": (st, [P, P, P, P]),
        "wedge_pr_pull_ordered": (st, [P, P, P, P]),
        "wedge_pr_order": (st, [P, P, P]),
        "wedge_trim_memory": (st, [i32]),
        "wedge_csc_relabel_by_degree": (st, [u32, u64, P, P, P, P, P, P, P, P, P]),
        "wedge_permute_rows": (st, [u32, u32, P, P, P, P]),
        "wedge_cc_labels_to_original": (st, [u32, P, P, P, P, P]),
        "wedge_selftest_timeout": (st, [i32]),
        "wedge_run_pr": (st, [P, P, u32, ctypes.c_float, ctypes.POINTER(wedge_opts),
                              ctypes.POINTER(wedge_stats), P]),
        "wedge_get_trace": (st, [P, ctypes.POINTER(wedge_iter_record), u32, ctypes.POINTER(u32)]),
        "wedge_graph_set_tuning": (st, [P, ctypes.POINTER(wedge_tuning)]),
        "wedge_run_bfs_batch": (st, [P, P, P, u32, u32, P, ctypes.POINTER(wedge_opts),
                                     ctypes.POINTER(wedge_stats), P]),
        "wedge_run_sssp_batch": (st, [P, P, P, u32, u32, P, ctypes.POINTER(wedge_opts),
                                     ctypes.POINTER(wedge_stats), P]),
        "wedge_run_bfs_batch_u8": (st, [P, P, P, u32, u32, P, ctypes.POINTER(wedge_opts),
                                        ctypes.POINTER(wedge_stats), P]),
        "wedge_mlp_forward": (st, [P, P, u32, P, P]),
        "wedge_mlp_forward_bf16": (st, [P, P, u32, P, P]),
        "wedge_mlp_loss_grad": (st, [P, P, P, u32, P, P, P]),
        "wedge_mlp_adam": (st, [P, P, P, P, u32, ctypes.c_float, P]),
        "wedge_set_cost_model": (st, [P, P]),
        "wedge_trace_candidates": (st, [P, i32, u32, ctypes.POINTER(wedge_opts), u32, P, P, P, u32,
                                        ctypes.POINTER(u32), P]),
        "wedge_graph_get_tuning": (st, [P, ctypes.POINTER(wedge_tuning)]),
        "wedge_kernel_launches": (u64, []),
        "wedge_last_error": (ctypes.c_char_p, []),
        "wedge_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise WedgeError(status, load().wedge_last_error().decode(errors="replace"))


def _ptr(x) -> int | None:
    """Data pointer of a torch tensor or numpy array (None passes NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    return int(x)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def wedge_default_opts(app) -> wedge_opts:
    o = wedge_opts()
    load().wedge_default_opts(APP_IDS[app] if isinstance(app, str) else int(app), ctypes.byref(o))
    return o


def wedge_graph_create(V, E, offsets, src, w=None, eidx_off=None, eidx=None, chunk_edges=32, stream=None):
    """Returns the opaque graph handle (int).  Arrays may live on the host
    (numpy) or the device (torch CUDA tensors, borrowed: keep them alive)."""
    h = ctypes.c_void_p()
    _check(load().wedge_graph_create(int(V), int(E), _ptr(offsets), _ptr(src), _ptr(w), _ptr(eidx_off),
                                     _ptr(eidx), int(chunk_edges), _stream(stream), ctypes.byref(h)))
    return h.value


def wedge_graph_destroy(handle):
    _check(load().wedge_graph_destroy(handle))


def wedge_graph_get_info(handle) -> dict:
    info = wedge_graph_info()
    _check(load().wedge_graph_get_info(handle, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


def wedge_graph_copy_edge_index(handle, eidx_off, eidx, stream=None):
    _check(load().wedge_graph_copy_edge_index(handle, _ptr(eidx_off), _ptr(eidx), _stream(stream)))


def wedge_graph_copy_edge_index_z(handle, zbo, zhdr, zwords, stream=None):
    _check(load().wedge_graph_copy_edge_index_z(handle, _ptr(zbo), _ptr(zhdr), _ptr(zwords), _stream(stream)))


def wedge_frontier_transform(handle, vertex_bitmap, log2_coarsen, chunk_list, chunk_count, stream=None):
    _check(load().wedge_frontier_transform(handle, _ptr(vertex_bitmap), int(log2_coarsen), _ptr(chunk_list),
                                           _ptr(chunk_count), _stream(stream)))


def wedge_frontier_transform_noalloc(V, E, eidx_off, eidx, vertex_bitmap, log2_coarsen, chunk_list, chunk_count,
                                     stream=None):
    """Allocation-free transformation for callers that cannot call cudaMalloc:
    its scratch is a fixed device array inside the library (see wedge.h)."""
    _check(load().wedge_frontier_transform_noalloc(int(V), int(E), _ptr(eidx_off), _ptr(eidx), _ptr(vertex_bitmap),
                                                   int(log2_coarsen), _ptr(chunk_list), _ptr(chunk_count),
                                                   _stream(stream)))


def wedge_frontier_transform_profile(handle, bitmap, k, schedule, chunk_list, chunk_count, stream=None):
    """Runs one transformation under `schedule` (0 library, 1 the paper's)
    and returns the per-warp records as an (n_warps, 2, 4) uint64 array:
    [warp, kernel, {start ns, end ns, busy cycles, SM}]."""
    import torch
    n = ctypes.c_uint32(0)
    _check(load().wedge_frontier_transform_profile(handle, None, int(k), int(schedule), None, None, None, 0,
                                                   ctypes.byref(n), _stream(stream)))
    stats = torch.zeros(n.value * 8, dtype=torch.int64, device=chunk_list.device)
    _check(load().wedge_frontier_transform_profile(handle, _ptr(bitmap), int(k), int(schedule), _ptr(chunk_list),
                                                   _ptr(chunk_count), _ptr(stats), n.value, ctypes.byref(n),
                                                   _stream(stream)))
    return stats.cpu().numpy().view(np.uint64).reshape(n.value, 2, 4)


def wedge_pull_iterate(handle, app, values, it, cur_bitmap, chunk_list, chunk_count, log2_coarsen, next_bitmap,
                       fullness, nfront, stream=None):
    a = APP_IDS[app] if isinstance(app, str) else int(app)
    _check(load().wedge_pull_iterate(handle, a, _ptr(values), int(it), _ptr(cur_bitmap), _ptr(chunk_list),
                                     _ptr(chunk_count), int(log2_coarsen), _ptr(next_bitmap), _ptr(fullness),
                                     _ptr(nfront), _stream(stream)))


def _opts(opts):
    return ctypes.byref(opts) if opts is not None else None


def wedge_run_bfs(handle, root, level, opts=None, want_stats=True, stream=None):
    st = wedge_stats()
    _check(load().wedge_run_bfs(handle, int(root), _ptr(level), _opts(opts),
                                ctypes.byref(st) if want_stats else None, _stream(stream)))
    return st if want_stats else None


def wedge_run_cc(handle, label, opts=None, want_stats=True, stream=None):
    st = wedge_stats()
    _check(load().wedge_run_cc(handle, _ptr(label), _opts(opts), ctypes.byref(st) if want_stats else None,
                               _stream(stream)))
    return st if want_stats else None


def wedge_run_sssp(handle, root, dist, opts=None, want_stats=True, stream=None):
    st = wedge_stats()
    _check(load().wedge_run_sssp(handle, int(root), _ptr(dist), _opts(opts),
                                 ctypes.byref(st) if want_stats else None, _stream(stream)))
    return st if want_stats else None


def wedge_run_pr(handle, rank, iters=20, damping=0.85, opts=None, want_stats=True, stream=None):
    st = wedge_stats()
    _check(load().wedge_run_pr(handle, _ptr(rank), int(iters), float(damping), _opts(opts),
                               ctypes.byref(st) if want_stats else None, _stream(stream)))
    return st if want_stats else None


def wedge_csc_relabel_by_degree(V, E, offsets, src, w, new_offsets, new_src, new_w, new_of_old, old_of_new=None,
                                stream=None):
    """Degree-ordered relabelling of a device CSC into the caller's device
    arrays (int32/uint32 torch tensors)."""
    _check(load().wedge_csc_relabel_by_degree(int(V), int(E), _ptr(offsets), _ptr(src), _ptr(w), _ptr(new_offsets),
                                              _ptr(new_src), _ptr(new_w), _ptr(new_of_old), _ptr(old_of_new),
                                              _stream(stream)))


def wedge_permute_rows(V, width, new_of_old, vals_in, vals_out, stream=None):
    """vals_out[v * width + c] = vals_in[new_of_old[v] * width + c] (32-bit words)."""
    _check(load().wedge_permute_rows(int(V), int(width), _ptr(new_of_old), _ptr(vals_in), _ptr(vals_out),
                                     _stream(stream)))


def wedge_cc_labels_to_original(V, old_of_new, labels, scratch, out, stream=None):
    """Component labels of a relabelled graph named by their smallest original id."""
    _check(load().wedge_cc_labels_to_original(int(V), _ptr(old_of_new), _ptr(labels), _ptr(scratch), _ptr(out),
                                              _stream(stream)))


def wedge_trim_memory(device=-1):
    """Returns the device memory kept by the library's pools to the driver."""
    _check(load().wedge_trim_memory(int(device)))


def wedge_selftest_timeout(kind):
    """Runs a device wait that cannot be satisfied; returns the library
    status (WEDGE_ERR_TIMEOUT = 4 is the expected outcome)."""
    return int(load().wedge_selftest_timeout(int(kind)))


def wedge_pr_pull(handle, contrib, sums, stream=None):
    """One PageRank in-edge pass: sums (int64 view of uint64, zeroed by the
    caller) = exact 2^-62 fixed-point in-edge sums of contrib (float32)."""
    _check(load().wedge_pr_pull(handle, _ptr(contrib), _ptr(sums), _stream(stream)))


def wedge_pr_order(handle, order, stream=None):
    """order (int32 device tensor of V): the position of each vertex's
    contribution in PageRank's gather order."""
    _check(load().wedge_pr_order(handle, _ptr(order), _stream(stream)))


def wedge_pr_pull_ordered(handle, contrib, sums, stream=None):
    """wedge_pr_pull on contributions already in the gather order."""
    _check(load().wedge_pr_pull_ordered(handle, _ptr(contrib), _ptr(sums), _stream(stream)))


def wedge_get_trace(handle, cap=1 << 16):
    buf = (wedge_iter_record * cap)()
    n = ctypes.c_uint32()
    _check(load().wedge_get_trace(handle, buf, cap, ctypes.byref(n)))
    return [{f: getattr(buf[i], f) for f, _ in wedge_iter_record._fields_} for i in range(min(n.value, cap))]


def wedge_graph_set_tuning(handle, dense_loader=0, blocks_per_sm=0, edge_index=0):
    t = wedge_tuning()
    t.dense_loader = int(dense_loader)
    t.blocks_per_sm = int(blocks_per_sm)
    t.edge_index = int(edge_index)
    _check(load().wedge_graph_set_tuning(handle, ctypes.byref(t)))


def wedge_graph_get_tuning(handle) -> dict:
    t = wedge_tuning()
    _check(load().wedge_graph_get_tuning(handle, ctypes.byref(t)))
    return {"dense_loader": t.dense_loader, "blocks_per_sm": t.blocks_per_sm, "edge_index": t.edge_index}


def wedge_run_bfs_batch(handle, roots, root_query, nqueries, levels, opts=None, want_stats=True, stream=None):
    """levels: device tensor of V * nqueries uint32 (vertex-major)."""
    r = np.ascontiguousarray(roots, dtype=np.uint32)
    q = None if root_query is None else np.ascontiguousarray(root_query, dtype=np.uint32)
    st = wedge_stats()
    _check(load().wedge_run_bfs_batch(handle, _ptr(r), _ptr(q), int(r.size), int(nqueries), _ptr(levels), _opts(opts),
                                      ctypes.byref(st) if want_stats else None, _stream(stream)))
    return st if want_stats else None


def wedge_run_bfs_batch_u8(handle, roots, root_query, nqueries, levels, opts=None, want_stats=True, stream=None):
    """levels: device tensor of V * nqueries uint8 (vertex-major, 0xFF unreached)."""
    r = np.ascontiguousarray(roots, dtype=np.uint32)
    q = None if root_query is None else np.ascontiguousarray(root_query, dtype=np.uint32)
    st = wedge_stats()
    _check(load().wedge_run_bfs_batch_u8(handle, _ptr(r), _ptr(q), int(r.size), int(nqueries), _ptr(levels),
                                         _opts(opts), ctypes.byref(st) if want_stats else None, _stream(stream)))
    return st if want_stats else None


def wedge_run_sssp_batch(handle, roots, root_query, nqueries, dist, opts=None, want_stats=True, stream=None):
    """dist: device tensor of V * nqueries uint32 (vertex-major)."""
    r = np.ascontiguousarray(roots, dtype=np.uint32)
    q = None if root_query is None else np.ascontiguousarray(root_query, dtype=np.uint32)
    st = wedge_stats()
    _check(load().wedge_run_sssp_batch(handle, _ptr(r), _ptr(q), int(r.size), int(nqueries), _ptr(dist), _opts(opts),
                                       ctypes.byref(st) if want_stats else None, _stream(stream)))
    return st if want_stats else None


def wedge_mlp_forward(params, x, n, y, stream=None):
    _check(load().wedge_mlp_forward(_ptr(params), _ptr(x), int(n), _ptr(y), _stream(stream)))


def wedge_mlp_forward_bf16(params, x, n, y, stream=None):
    _check(load().wedge_mlp_forward_bf16(_ptr(params), _ptr(x), int(n), _ptr(y), _stream(stream)))


def wedge_mlp_loss_grad(params, x, t, n, grad, loss, stream=None):
    _check(load().wedge_mlp_loss_grad(_ptr(params), _ptr(x), _ptr(t), int(n), _ptr(grad), _ptr(loss),
                                      _stream(stream)))


def wedge_mlp_adam(params, grad, m, v, step, lr, stream=None):
    _check(load().wedge_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr), _stream(stream)))


def wedge_set_learned_band(handle, lo, hi):
    _check(load().wedge_set_learned_band(handle, float(lo), float(hi)))


def wedge_set_cost_model(handle, params):
    """params: FP32 array of MLP_PARAMS (host numpy or device tensor), or None."""
    if params is not None and isinstance(params, np.ndarray):
        params = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().wedge_set_cost_model(handle, _ptr(params)))


def wedge_trace_candidates(handle, app, root=0, opts=None, max_iters=0, cap=4096, stream=None):
    """Returns (features [n, 6, 12], ms [n, 6], chosen [n]) as numpy arrays."""
    a = APP_IDS[app] if isinstance(app, str) else int(app)
    feat = np.zeros((cap, MLP_CANDIDATES, MLP_FEATURES), dtype=np.float32)
    ms = np.zeros((cap, MLP_CANDIDATES), dtype=np.float32)
    chosen = np.zeros(cap, dtype=np.uint32)
    n = ctypes.c_uint32()
    _check(load().wedge_trace_candidates(handle, a, int(root), _opts(opts), int(max_iters), feat.ctypes.data,
                                         ms.ctypes.data, chosen.ctypes.data, int(cap), ctypes.byref(n),
                                         _stream(stream)))
    k = n.value
    return feat[:k].copy(), ms[:k].copy(), chosen[:k].copy()


def wedge_kernel_launches() -> int:
    return int(load().wedge_kernel_launches())


def wedge_last_error() -> str:
    return load().wedge_last_error().decode(errors="replace")


def wedge_version() -> str:
    return load().wedge_version().decode()


class Graph:
    """Owns a graph handle plus the device tensors it borrows.

    ``Graph.from_csc(g)`` uploads any object with V, offsets, src and
    optional w (numpy, CSC order) as torch CUDA tensors."""

    def __init__(self, handle, keep=()):
        self.handle = handle
        self._keep = list(keep)
        self.info = wedge_graph_get_info(handle)

    @classmethod
    def from_csc(cls, g, device="cuda", with_weights=True, stream=None):
        import torch
        off = torch.from_numpy(np.ascontiguousarray(g.offsets, dtype=np.uint32).view(np.int32)).to(device)
        src = torch.from_numpy(np.ascontiguousarray(g.src, dtype=np.uint32).view(np.int32)).to(device)
        w = None
        if with_weights and getattr(g, "w", None) is not None:
            w = torch.from_numpy(np.ascontiguousarray(g.w, dtype=np.uint32).view(np.int32)).to(device)
        h = wedge_graph_create(g.V, src.numel(), off, src, w, stream=stream)
        return cls(h, keep=(off, src, w))

    @property
    def device_src(self):
        """The device tensor of the in-edge sources (int32 view), or None
        when the graph was created from a raw handle."""
        return self._keep[1] if len(self._keep) > 1 else None

    @property
    def V(self):
        return self.info["V"]

    @property
    def E(self):
        return self.info["E"]

    def close(self):
        if self.handle:
            wedge_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
