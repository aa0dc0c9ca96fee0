"""Helpers for the GPU parity tests (device upload, bitmaps)."""
import numpy as np
import torch

from paper_1903_07754_gb300 import wedge

INF = 0xFFFFFFFF


def u32(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def dev_u32(a) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def empty_u32(n: int) -> torch.Tensor:
    return torch.empty(max(int(n), 1), dtype=torch.int32, device="cuda")


def zeros_u32(n: int) -> torch.Tensor:
    return torch.zeros(max(int(n), 1), dtype=torch.int32, device="cuda")


def bitmap(V: int, members) -> np.ndarray:
    """uint32 words with bit (v & 31) of word v >> 5 set for each member
    (member ids, or a V-long boolean mask)."""
    m = np.asarray(members)
    mask = np.zeros(V, dtype=bool)
    if m.dtype == bool:
        mask[:] = m
    elif m.size:
        mask[m.astype(np.int64)] = True
    bits = np.zeros(((V + 31) // 32) * 32, dtype=np.uint64)
    bits[:V] = mask
    return (bits.reshape(-1, 32) << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)


def unpack(words: np.ndarray, V: int) -> np.ndarray:
    w = words.astype(np.uint64)
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)).astype(bool).reshape(-1)
    return bits[:V]


def graph(g, with_weights=True) -> wedge.Graph:
    return wedge.Graph.from_csc(g, with_weights=with_weights)


def opts(app, switch=None, tau=None, k=None, trace=0, max_iters=0):
    o = wedge.wedge_default_opts(app)
    if switch is not None:
        o.switch_mode = switch
    if tau is not None:
        o.tau_bp = tau
    if k is not None:
        o.log2_coarsen = k
    o.trace = trace
    o.max_iters = max_iters
    return o
