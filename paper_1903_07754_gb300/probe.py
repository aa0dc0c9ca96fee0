"""ctypes binding of libwedge_probe.so (include/wedge_probe.h): a
measurement tool for the benchmark, not part of the engine.  Raises if the
library cannot be loaded."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwedge_probe.so")
EXPORTS = ["wedge_probe_gather"]

_lib = None


def load(path: str = LIB_PATH):
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.wedge_probe_gather.restype = ctypes.c_int
    lib.wedge_probe_gather.argtypes = [P, ctypes.c_uint64, P, P, ctypes.c_uint32, P]
    _lib = lib
    return lib


def wedge_probe_gather(src, E, vals, sink, blocks_per_sm=4, stream=None):
    """src: E uint32 sources (int32 device tensor, 16-byte aligned); vals:
    float32 device tensor; sink: 1 float32 device tensor.  Runs on torch's
    current stream unless `stream` (a torch stream) is given."""
    import torch
    s = (stream or torch.cuda.current_stream()).cuda_stream
    rc = load().wedge_probe_gather(src.data_ptr() if E else None, int(E), vals.data_ptr(), sink.data_ptr(),
                                   int(blocks_per_sm), s)
    if rc != 0:
        raise RuntimeError(f"wedge_probe_gather: CUDA error {rc}")
