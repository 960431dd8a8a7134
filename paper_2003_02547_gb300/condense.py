"""Partial condensing through the C ABI (gq_condense_dims, gq_condense,
gq_condense_device, gq_expand): argument marshalling only, the condensing
runs in libgq (host) or in its CUDA kernel (device)."""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from . import gq
from .batch import QpBatch


def condensed_dims(src: QpBatch, i: int, block: int) -> np.ndarray:
    lib = gq.load()
    n = ctypes.c_size_t()
    gq.check(lib.gq_condense_dims(src.h, int(i), int(block), None, 0, ctypes.byref(n)))
    d = np.zeros(n.value, dtype=np.int32)
    gq.check(lib.gq_condense_dims(src.h, int(i), int(block), d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  d.size, ctypes.byref(n)))
    return d


def condense(src: QpBatch, indices: Sequence[int], block: int, device: str = "cuda") -> QpBatch:
    """A new batch holding QPs ``indices`` of ``src`` condensed by ``block``."""
    dims = [condensed_dims(src, i, block) for i in indices]
    dst = QpBatch(None, device=device, dims=dims)
    lib = gq.load()
    for k, i in enumerate(indices):
        gq.check(lib.gq_condense(src.h, int(i), int(block), dst.h, k))
    return dst


def condense_device(src: QpBatch, block: int, stream=None, host_copy: bool = True) -> QpBatch:
    """Every QP of the uploaded batch ``src`` condensed by ``block`` on the
    device: a new batch whose device data the condensing kernel writes.  With
    ``host_copy`` the condensed data are also copied to its host staging (for
    the host getters); the copy synchronises the stream."""
    import torch
    lib = gq.load()
    dims = [condensed_dims(src, i, block) for i in range(src.nqp)]
    dst = QpBatch(None, device=src.device, dims=dims)
    dst.upload(stream)
    nbytes = int(lib.gq_condense_ws_bytes(src.h, int(block)))
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=src.device)
    gq.check(lib.gq_condense_device(src.h, int(block), dst.h, ws.data_ptr(), nbytes, src.stream_ptr(stream)))
    dst._condense_ws = ws   # kept alive with the batch until the kernel has run
    if host_copy:
        torch.cuda.synchronize()
        dst.host_in._np[dst.host_in.off:dst.host_in.off + dst.sizes.in_bytes] = \
            dst.dev_in[:dst.sizes.in_bytes].cpu().numpy()
    return dst


def expand(src: QpBatch, i: int, block: int, dst: QpBatch, k: int, sol=None):
    """(y, pi, lam, t) of QP i of ``src`` from the condensed solution of QP k
    of ``dst`` (default: dst's host solution buffer)."""
    lib = gq.load()
    y2, pi2, lam2, t2 = [np.ascontiguousarray(a, dtype=np.float64) for a in (sol or dst.solution(k))]
    o = src.offsets(i)
    y, pi, lam, t = (np.zeros(int(o[4])), np.zeros(int(o[5])), np.zeros(int(o[6])), np.zeros(int(o[7])))
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    gq.check(lib.gq_expand(src.h, int(i), int(block), dst.h, int(k), P(y2), P(pi2), P(lam2), P(t2),
                           P(y), P(pi), P(lam), P(t)))
    return y, pi, lam, t
