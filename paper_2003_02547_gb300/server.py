"""Python handle of the continuous-batching server (include/gq_server.h).

Argument marshalling only: admission, micro-batch assembly, the resident
warm-start cache, the lanes' streams and the solves all run in libgq's native
worker thread and CUDA kernels.  The device and pinned arenas are PyTorch
allocations owned here and lent to the library.
"""
from __future__ import annotations

import ctypes
import time
from typing import Dict, Optional, Tuple

import numpy as np

from . import gq


class Server:
    def __init__(self, budget_bytes: int, lanes: int = 4, max_batch: int = 256, max_wait_us: int = 0,
                 cache_bytes: Optional[int] = None, pinned_bytes: Optional[int] = None,
                 arg: Optional[gq.IpmArg] = None, device: int = 0, class_ratio: Optional[float] = None):
        import torch
        self.lib = gq.load()
        cfg = gq.ServerCfg()
        gq.check(self.lib.gq_server_cfg_default(ctypes.byref(cfg)))
        cfg.lanes = lanes
        cfg.max_batch = max_batch
        cfg.max_wait_us = max_wait_us
        cfg.device = device
        if cache_bytes is None:
            cache_bytes = budget_bytes // 4
        cfg.cache_bytes = int(cache_bytes)
        if arg is not None:
            cfg.arg = arg
        if class_ratio is not None:
            cfg.class_ratio = float(class_ratio)
        self.cfg = cfg
        if pinned_bytes is None:
            # inputs + solutions of one lane are a small part of its device share
            pinned_bytes = min(int(budget_bytes - cache_bytes), 1 << 30)
        self.dev_arena = torch.empty(int(budget_bytes), dtype=torch.uint8, device=f"cuda:{device}")
        self.pinned = torch.empty(int(pinned_bytes), dtype=torch.uint8).pin_memory()
        h = ctypes.c_void_p()
        gq.check(self.lib.gq_server_create(ctypes.byref(cfg), self.dev_arena.data_ptr(), int(budget_bytes),
                                           self.pinned.data_ptr(), int(pinned_bytes), ctypes.byref(h)))
        self.h = h
        self._out: Dict[int, Tuple] = {}
        self._keep: Dict[int, object] = {}

    def submit(self, src, i: int, key: int = 0, warm: bool = False, t_arrival_ns: int = 0,
               outputs: bool = True) -> int:
        """Queue QP ``i`` of the host-staged batch ``src`` (a QpBatch)."""
        req = gq.Request()
        req.src = src.h
        req.src_qp = int(i)
        req.warm = 1 if warm else 0
        req.key = int(key)
        req.t_arrival_ns = int(t_arrival_ns)
        out = None
        if outputs:
            o = src.offsets(i)
            out = (np.empty(int(o[4])), np.empty(int(o[5])), np.empty(int(o[6])), np.empty(int(o[7])))
            P = ctypes.POINTER(ctypes.c_double)
            req.y, req.pi, req.lam, req.t = (a.ctypes.data_as(P) for a in out)
        tk = ctypes.c_int64()
        gq.check(self.lib.gq_server_submit(self.h, ctypes.byref(req), ctypes.byref(tk)))
        t = int(tk.value)
        if out is not None:
            self._out[t] = out
        self._keep[t] = src
        return t

    def poll(self, ticket: int) -> gq.TicketInfo:
        info = gq.TicketInfo()
        gq.check(self.lib.gq_server_poll(self.h, int(ticket), ctypes.byref(info)))
        return info

    def result(self, ticket: int):
        """(info, (y, pi, lam, t) or None) of a finished ticket; releases it."""
        info = self.poll(ticket)
        if not info.done:
            raise RuntimeError(f"ticket {ticket} not done")
        self._keep.pop(ticket, None)
        return info, self._out.pop(ticket, None)

    def drain(self, timeout_s: float = 60.0) -> None:
        gq.check(self.lib.gq_server_drain(self.h, int(timeout_s * 1e9)))

    def report(self) -> Dict[str, int]:
        r = gq.ServerReport()
        gq.check(self.lib.gq_server_report_get(self.h, ctypes.byref(r)))
        return {name: int(getattr(r, name)) for name, _ in gq.ServerReport._fields_}

    def close(self) -> None:
        if self.h is not None:
            gq.check(self.lib.gq_server_destroy(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def now_ns() -> int:
    """The clock the server timestamps with (CLOCK_MONOTONIC)."""
    return time.monotonic_ns()
