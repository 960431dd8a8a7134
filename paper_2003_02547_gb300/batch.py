"""Batch builder over the gq C ABI.

Marshals a list of OCP QPs into the caller-owned buffers the library needs
(host handle memory, pinned host staging, device buffers from PyTorch) and
calls the C entry points.  No solver arithmetic happens here.
"""
from __future__ import annotations

import ctypes
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import gq


def _ptr(a: Optional[np.ndarray], ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def dims_of(qps: Sequence) -> np.ndarray:
    out: List[int] = []
    for qp in qps:
        out.append(qp.N)
        for n in range(qp.N + 1):
            out += [qp.nx[n], qp.nu[n], qp.nbx(n), qp.nbu(n), qp.ng(n)]
    return np.array(out, dtype=np.int32)


def ns_of(qps: Sequence) -> Optional[np.ndarray]:
    """Slack pairs per stage (soft constraints, Sec. 2.2), or None if no QP
    has any."""
    out = [qp.ns(n) if hasattr(qp, "ns") else 0 for qp in qps for n in range(qp.N + 1)]
    return np.array(out, dtype=np.int32) if any(out) else None


def slots_of(qps: Sequence) -> np.ndarray:
    """Stages whose ``stage_key`` is equal (and not None) share a data block."""
    ids: Dict[object, int] = {}
    out = []
    for qp in qps:
        keys = qp.stage_key if qp.stage_key else [None] * (qp.N + 1)
        for n in range(qp.N + 1):
            k = keys[n]
            if k is None:
                out.append(-1)
            else:
                out.append(ids.setdefault(k, len(ids)))
    return np.array(out, dtype=np.int32)


class HostBuffer:
    """Host memory for the library: pinned torch storage when CUDA is usable,
    else an aligned numpy array."""

    def __init__(self, nbytes: int, pinned: bool):
        self.nbytes = int(nbytes)
        n = max(self.nbytes, 1) + 256
        if pinned:
            import torch
            self._t = torch.empty(n, dtype=torch.uint8, pin_memory=True)
            base = self._t.data_ptr()
            self._np = self._t.numpy()
        else:
            self._t = None
            self._np = np.zeros(n, dtype=np.uint8)
            base = self._np.ctypes.data
        self.off = (-base) % 256
        self.ptr = base + self.off

    def view(self, dtype, offset_bytes: int, count: int) -> np.ndarray:
        itemsize = np.dtype(dtype).itemsize
        start = self.off + offset_bytes
        return self._np[start:start + count * itemsize].view(dtype)


class QpBatch:
    """A batch of OCP QPs laid out for the GPU solver.

    ``device`` is a torch device string; ``share`` turns equal stage keys into
    one shared data block.  Problem data are written with the C setters.
    """

    def __init__(self, qps: Optional[Sequence], device: str = "cuda", share: bool = True, pinned: bool = True,
                 set_data: bool = True, dims: Optional[Sequence[np.ndarray]] = None):
        """``qps``: OcpQp objects; or None with ``dims``, one dims array per QP
        (the C ABI format: N, then nx, nu, nbx, nbu, ng per stage), for a batch
        whose data the caller writes through the C setters."""
        self.lib = gq.load()
        if qps is None:
            self.qps = None
            self.nqp = len(dims)
            self.dims = np.ascontiguousarray(np.concatenate([np.asarray(d, dtype=np.int32) for d in dims]))
            self.slots = None
            self.stage_ns = None
            set_data = False
        else:
            self.qps = list(qps)
            self.nqp = len(self.qps)
            self.dims = dims_of(self.qps)
            self.slots = slots_of(self.qps) if share else None
            self.stage_ns = ns_of(self.qps)
        slot_p = _ptr(self.slots, ctypes.c_int) if self.slots is not None else None
        mem = self.lib.gq_batch_memsize(self.nqp, _ptr(self.dims, ctypes.c_int), self.dims.size, slot_p)
        if mem == 0:
            gq.check(gq.GQ_ERR_DIMS)
        self._hmem = np.zeros(mem + 64, dtype=np.uint8)
        base = self._hmem.ctypes.data
        self._hmem_ptr = base + ((-base) % 64)
        h = ctypes.c_void_p()
        ns_p = _ptr(self.stage_ns, ctypes.c_int) if self.stage_ns is not None else None
        gq.check(self.lib.gq_batch_create_soft(self.nqp, _ptr(self.dims, ctypes.c_int), self.dims.size, slot_p,
                                               ns_p, self._hmem_ptr, mem, ctypes.byref(h)))
        self.h = h
        self.sizes = gq.Sizes()
        gq.check(self.lib.gq_batch_sizes(self.h, ctypes.byref(self.sizes)))
        self.device = device
        use_cuda = device is not None and device.startswith("cuda")
        self.host_in = HostBuffer(self.sizes.in_bytes, pinned and use_cuda)
        self.host_sol = HostBuffer(self.sizes.sol_bytes, pinned and use_cuda)
        if use_cuda:
            import torch
            self.dev_in = torch.empty(max(self.sizes.in_bytes, 256), dtype=torch.uint8, device=device)
            self.dev_sol = torch.zeros(max(self.sizes.sol_bytes, 256), dtype=torch.uint8, device=device)
            self.dev_ws = torch.zeros(max(self.sizes.ws_bytes, 256), dtype=torch.uint8, device=device)
            dptr = (self.dev_in.data_ptr(), self.dev_sol.data_ptr(), self.dev_ws.data_ptr())
        else:
            # host-only use (layout and setters): placeholders never dereferenced
            self._fake = [HostBuffer(256, False) for _ in range(3)]
            dptr = tuple(f.ptr for f in self._fake)
        gq.check(self.lib.gq_batch_attach(self.h, self.host_in.ptr, self.host_sol.ptr, *dptr))
        if set_data:
            self.set_all()

    # ---------------- setters ----------------
    def set_qp(self, i: int, qp, done_slots: Optional[set] = None, first_stage: int = 0) -> None:
        L = self.lib
        h = self.h
        base = self._stage_base(i)
        for n in range(qp.N + 1):
            if done_slots is not None and self.slots is not None:
                s = int(self.slots[base + n])
                if s >= 0:
                    if s in done_slots:
                        continue
                    done_slots.add(s)
            nx, nu = qp.nx[n], qp.nu[n]
            if n < qp.N:
                A, B, b = _f64(qp.A[n]), _f64(qp.B[n]), _f64(qp.b[n])
                gq.check(L.gq_set_dynamics(h, i, n, _ptr(A), max(A.shape[0], 1), _ptr(B), max(B.shape[0], 1),
                                           _ptr(b)))
            Q, S, R = _f64(qp.Q[n]), _f64(qp.S[n]), _f64(qp.R[n])
            q, r = _f64(qp.q[n]), _f64(qp.r[n])
            gq.check(L.gq_set_cost(h, i, n, _ptr(Q), max(nx, 1), _ptr(S), max(nu, 1), _ptr(R), max(nu, 1),
                                   _ptr(q), _ptr(r)))
            ibu, ibx = _i32(qp.idxbu[n]), _i32(qp.idxbx[n])
            gq.check(L.gq_set_box(h, i, n, _ptr(ibu, ctypes.c_int), _ptr(_f64(qp.lbu[n])), _ptr(_f64(qp.ubu[n])),
                                  _ptr(ibx, ctypes.c_int), _ptr(_f64(qp.lbx[n])), _ptr(_f64(qp.ubx[n]))))
            ng = qp.ng(n)
            if ng:
                C, D = _f64(qp.C[n]), _f64(qp.D[n])
                gq.check(L.gq_set_general(h, i, n, _ptr(C), ng, _ptr(D), ng, _ptr(_f64(qp.lg[n])),
                                          _ptr(_f64(qp.ug[n]))))
            if hasattr(qp, "ns") and qp.ns(n):
                gq.check(L.gq_set_soft(h, i, n, _ptr(_i32(qp.idxs[n]), ctypes.c_int), _ptr(_f64(qp.Zl[n])),
                                       _ptr(_f64(qp.Zu[n])), _ptr(_f64(qp.zl[n])), _ptr(_f64(qp.zu[n])),
                                       _ptr(_f64(qp.lls[n])), _ptr(_f64(qp.lus[n]))))

    def _stage_base(self, i: int) -> int:
        if not hasattr(self, "_sbase"):
            acc = 0
            self._sbase = []
            for qp in self.qps:
                self._sbase.append(acc)
                acc += qp.N + 1
        return self._sbase[i]

    def horizon(self, i: int) -> int:
        pos = 0
        for q in range(i):
            pos += 1 + 5 * (int(self.dims[pos]) + 1)
        return int(self.dims[pos])

    def stage_dims(self, i: int):
        """[(nx, nu, nbx, nbu, ng)] of QP i, from the dims array."""
        pos = 0
        for q in range(i):
            pos += 1 + 5 * (int(self.dims[pos]) + 1)
        N = int(self.dims[pos])
        d = self.dims[pos + 1:pos + 1 + 5 * (N + 1)].reshape(N + 1, 5)
        return [tuple(int(v) for v in row) for row in d]

    def to_ocp(self, i: int):
        """QP i as an OcpQp, read back from the staged data with the C getters
        (for checking data written by C routines such as gq_condense)."""
        from .workloads import OcpQp
        L, h = self.lib, self.h
        sd = self.stage_dims(i)
        N = len(sd) - 1
        nx = [d[0] for d in sd]
        nu = [d[1] for d in sd]
        f = lambda r, c: np.zeros((max(r, 1), max(c, 1)), order="F")
        P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        PI = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        out = {k: [] for k in ("A", "B", "b", "Q", "S", "R", "q", "r", "idxbu", "lbu", "ubu", "idxbx", "lbx", "ubx",
                               "C", "D", "lg", "ug")}
        soft: dict = {}
        for n in range(N + 1):
            x, u, nbx, nbu, ng = sd[n]
            if n < N:
                x1 = nx[n + 1]
                A, B, bv = f(x1, x), f(x1, u), np.zeros(max(x1, 1))
                gq.check(L.gq_get_dynamics(h, i, n, P(A), max(x1, 1), P(B), max(x1, 1), P(bv)))
                out["A"].append(A[:x1, :x].copy())
                out["B"].append(B[:x1, :u].copy())
                out["b"].append(bv[:x1].copy())
            Q, S, R, q, r = f(x, x), f(u, x), f(u, u), np.zeros(max(x, 1)), np.zeros(max(u, 1))
            gq.check(L.gq_get_cost(h, i, n, P(Q), max(x, 1), P(S), max(u, 1), P(R), max(u, 1), P(q), P(r)))
            out["Q"].append(Q[:x, :x].copy())
            out["S"].append(S[:u, :x].copy())
            out["R"].append(R[:u, :u].copy())
            out["q"].append(q[:x].copy())
            out["r"].append(r[:u].copy())
            ibu, ibx = np.zeros(max(nbu, 1), dtype=np.int32), np.zeros(max(nbx, 1), dtype=np.int32)
            lbu, ubu, lbx, ubx = (np.zeros(max(k, 1)) for k in (nbu, nbu, nbx, nbx))
            gq.check(L.gq_get_box(h, i, n, PI(ibu), P(lbu), P(ubu), PI(ibx), P(lbx), P(ubx)))
            out["idxbu"].append(ibu[:nbu].astype(np.int64))
            out["lbu"].append(lbu[:nbu].copy())
            out["ubu"].append(ubu[:nbu].copy())
            out["idxbx"].append(ibx[:nbx].astype(np.int64))
            out["lbx"].append(lbx[:nbx].copy())
            out["ubx"].append(ubx[:nbx].copy())
            C, D, lg, ug = f(ng, x), f(ng, u), np.zeros(max(ng, 1)), np.zeros(max(ng, 1))
            gq.check(L.gq_get_general(h, i, n, P(C), max(ng, 1), P(D), max(ng, 1), P(lg), P(ug)))
            out["C"].append(C[:ng, :x].copy())
            out["D"].append(D[:ng, :u].copy())
            out["lg"].append(lg[:ng].copy())
            out["ug"].append(ug[:ng].copy())
            nsv = ctypes.c_int()
            gq.check(L.gq_get_soft(h, i, n, ctypes.byref(nsv), None, None, None, None, None, None, None))
            ns = nsv.value
            arrs = [np.zeros(max(ns, 1), dtype=np.int32)] + [np.zeros(max(ns, 1)) for _ in range(6)]
            if ns:
                gq.check(L.gq_get_soft(h, i, n, None, PI(arrs[0]), *[P(a) for a in arrs[1:]]))
            for key, a in zip(("idxs", "Zl", "Zu", "zl", "zu", "lls", "lus"), arrs):
                soft.setdefault(key, []).append(a[:ns].copy())
        if any(len(v) for v in soft.get("idxs", [])):
            out.update(soft)
        qp = OcpQp(N=N, nx=nx, nu=nu, **out)
        qp.validate()
        return qp

    def set_all(self) -> None:
        done: set = set()
        for i, qp in enumerate(self.qps):
            self.set_qp(i, qp, done)

    def replace_qp(self, i: int, qp) -> None:
        """Rewrite the stage data of QP i that no other stage shares (for
        example the x0-dependent stage 0 after a new measurement)."""
        self.qps[i] = qp
        shared = set()
        if self.slots is not None:
            vals, counts = np.unique(self.slots[self.slots >= 0], return_counts=True)
            shared = set(int(v) for v, c in zip(vals, counts) if c > 1)
        self.set_qp(i, qp, done_slots=shared if self.slots is not None else None)

    # ---------------- device calls ----------------
    def stream_ptr(self, stream=None) -> int:
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return s.cuda_stream

    def upload(self, stream=None) -> None:
        gq.check(self.lib.gq_upload(self.h, self.stream_ptr(stream)))

    def upload_sol(self, stream=None) -> None:
        gq.check(self.lib.gq_upload_sol(self.h, self.stream_ptr(stream)))

    def solve(self, arg: gq.IpmArg, stream=None) -> None:
        gq.check(self.lib.gq_solve(self.h, ctypes.byref(arg), self.stream_ptr(stream)))

    def download(self, stream=None) -> None:
        gq.check(self.lib.gq_download(self.h, self.stream_ptr(stream)))

    def residuals(self, stream=None) -> None:
        gq.check(self.lib.gq_residuals(self.h, self.stream_ptr(stream)))

    def newton_step(self, arg: gq.IpmArg, sigma_mu: float, dev_dir, stream=None) -> None:
        gq.check(self.lib.gq_newton_step(self.h, ctypes.byref(arg), float(sigma_mu), dev_dir.data_ptr(),
                                         self.stream_ptr(stream)))

    # ---------------- schedule ----------------
    def schedule(self) -> gq.Schedule:
        sch = gq.Schedule()
        gq.check(self.lib.gq_get_schedule(self.h, ctypes.byref(sch)))
        return sch

    def set_schedule(self, warp_max_nv: int, block_threads: int = 0, tensor_cores: int = 1) -> None:
        sch = gq.Schedule(warp_max_nv, block_threads, 0, 0, tensor_cores)
        gq.check(self.lib.gq_set_schedule(self.h, ctypes.byref(sch)))

    def autotune(self, arg: gq.IpmArg, reps: int = 2, stream=None):
        """Pick the fastest schedule by timing solves; returns (schedule, ms)."""
        sch = gq.Schedule()
        ms = ctypes.c_double()
        gq.check(self.lib.gq_autotune(self.h, ctypes.byref(arg), self.stream_ptr(stream), int(reps),
                                      ctypes.byref(sch), ctypes.byref(ms)))
        return sch, ms.value

    # ---------------- results ----------------
    def stats(self, i: int) -> gq.Stats:
        s = gq.Stats()
        gq.check(self.lib.gq_get_stats(self.h, i, ctypes.byref(s)))
        return s

    def all_stats(self) -> np.ndarray:
        """Structured array of per-QP stats from the host sol buffer."""
        dt = np.dtype([("status", "<i4"), ("iters", "<i4"), ("flags", "<i4"), ("ir_total", "<i4"),
                       ("n_fact", "<i4"), ("n_fact64", "<i4"), ("n_solve", "<i4"), ("n_res", "<i4"),
                       ("res", "<f8", 4)])
        return self.host_sol.view(dt, 0, self.nqp).copy()

    def offsets(self, i: int) -> np.ndarray:
        off = (ctypes.c_int64 * 8)()
        gq.check(self.lib.gq_get_sol_offsets(self.h, i, off))
        return np.array(off[:], dtype=np.int64)

    def solution(self, i: int, buf: Optional[np.ndarray] = None):
        """(y, pi, lam, t) of QP i from a sol-layout float64 array (default:
        the host sol buffer)."""
        if buf is None:
            buf = self.host_sol.view(np.float64, 0, self.sizes.sol_bytes // 8)
        o = self.offsets(i)
        return (buf[o[0]:o[0] + o[4]].copy(), buf[o[1]:o[1] + o[5]].copy(),
                buf[o[2]:o[2] + o[6]].copy(), buf[o[3]:o[3] + o[7]].copy())

    def set_guess(self, i: int, y=None, pi=None, lam=None, t=None) -> None:
        gq.check(self.lib.gq_set_guess(self.h, i, _ptr(_f64(y)) if y is not None else None,
                                       _ptr(_f64(pi)) if pi is not None else None,
                                       _ptr(_f64(lam)) if lam is not None else None,
                                       _ptr(_f64(t)) if t is not None else None))
