"""Benchmark: batched OCP-QP IPM solves per second on GB300.

Workload (one "step"): the mass-spring chain of Sec. 5.1 with 8 masses
(nx = 16, nu = 7), N = 30, Q = I, R = I, |u| <= 0.5, |x| <= 4; a batch of
1024 QPs that differ only in x0 ~ U[-1, 1]^16, each solved to KKT residual
1e-8 by the mixed-precision IPM (FP32 Riccati factor/solve; residual
mat-vecs in double-float on the FP32 pipe, about 48 bits; FP64 refinement
updates, recovery, step length and duality measure) in one kernel launch.

Prints one JSON line: the metric, its end-to-end counterpart through the C
ABI with host buffers, the roofline of the timed kernel (algorithmic flops of
the flop model below over its CUDA-event time, against the flop-mix-weighted
ALU peak), the sampled SM clocks, the plain per-QP FP64 GPU baseline and the
CPU oracle on a bounded sample.  ``--impl reference`` times the CPU oracle
instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "QP solves/s to KKT res 1e-8 (mixed+batched vs plain FP64 GPU IPM); p50/p99 ms"
UNIT = "QP/s"
BATCH = 1024
HORIZON = 30
MASSES = 8
WORKLOAD = "mass-spring chain M=8 (nx=16, nu=7), N=30, batch 1024, x0~U[-1,1]"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gq", choices=["gq", "reference"])
    p.add_argument("--batch", type=int, default=BATCH)
    p.add_argument("--plain-sample", type=int, default=64,
                   help="QPs solved one launch each for the plain FP64 GPU baseline")
    p.add_argument("--cpu-sample", type=int, default=48, help="QPs in the oracle CPU baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the serving run and the ragged / large-stage batch measurements")
    p.add_argument("--serving-rate", type=float, default=20000.0, help="offered load of the serving run (QP/s)")
    p.add_argument("--serving-duration", type=float, default=0.5, help="seconds of Poisson arrivals")
    return p.parse_args()


# ----------------------------------------------------------------------------
# flop model: algorithmic work per QP (stage products, Cholesky, triangular
# solves and residual mat-vecs of the square-root Riccati IPM)
# ----------------------------------------------------------------------------
def qp_flops(qp):
    """(factorisation, one Riccati solve, one residual evaluation) flops."""
    f = s = r = 0.0
    for n in range(qp.N + 1):
        nv = qp.nx[n] + qp.nu[n]
        nx1 = qp.nx[n + 1] if n < qp.N else 0
        ng = qp.ng(n)
        f += nx1 * nx1 * nv + nx1 * nv * nv + nv ** 3 / 3.0 + ng * nv * nv
        s += 2.0 * (nv * nv + 2.0 * nx1 * nv)
        r += 2.0 * (nv * nv + 2.0 * nx1 * nv + 2.0 * ng * nv)
    return f, s, r


# ALU peaks (flop/s): measured on the device by the library's FMA probe
# (gq_probe_fma_rate) when the bench starts; the nominal figures below are
# kept for reference and used only if the probe fails
P32_NOMINAL = 152 * 128 * 2 * 2.07e9   # FP32 FMA lanes x 2 x max SM clock
P64_NOMINAL = 1.25e12                  # nominal GB300 FP64 rate
PEAKS = {"fp32": P32_NOMINAL, "fp64": P64_NOMINAL, "source": "nominal"}


def measure_peaks(stream_ptr) -> None:
    import ctypes
    from paper_2003_02547_gb300 import gq
    lib = gq.load()
    f32, f64 = ctypes.c_double(), ctypes.c_double()
    if lib.gq_probe_fma_rate(0, stream_ptr, ctypes.byref(f32)) == 0 and \
            lib.gq_probe_fma_rate(1, stream_ptr, ctypes.byref(f64)) == 0 and f32.value > 0 and f64.value > 0:
        PEAKS.update(fp32=f32.value, fp64=f64.value, source="measured (FMA probe, gq_probe_fma_rate)")


# FP32 instructions per double-float multiply-add (the kernel's df_acc: three
# FMAs, one multiply and eight adds), against one FP32 FMA for the same two
# algorithmic flops: double-float work runs at 1/12 of the FP32 flop rate
DF_COST = 12.0


def t_min_of(f32, f64, fdf):
    """Shortest time of the work at the measured ALU peaks, each class on the
    unit that executes it."""
    return f32 / PEAKS["fp32"] + f64 / PEAKS["fp64"] + fdf * DF_COST / PEAKS["fp32"]


def alu_roofline(qps, stats, seconds, warp_max_nv: int = 32):
    """Achieved algorithmic flop rates of one batch solve and their fraction
    of the flop-mix-weighted ALU peak (FP32 lanes for the FP32 work, the FP64
    rate for the FP64 work, FP32 lanes / DF_COST for the double-float work)."""
    f32, f64, fdf = work_split(qps, stats, warp_max_nv)
    t_min = t_min_of(f32, f64, fdf)
    return {"fp32_tflops": f32 / seconds / 1e12, "fp64_tflops": f64 / seconds / 1e12,
            "df_tflops": fdf / seconds / 1e12,
            "fp32_frac_of_peak": f32 / seconds / PEAKS["fp32"], "fp64_frac_of_peak": f64 / seconds / PEAKS["fp64"],
            "frac_of_mix_peak": t_min / seconds if t_min > 0 else None}


def in_warp_kernel(qp, warp_max_nv: int = 32) -> bool:
    """The schedule's one-warp bucket: every stage with nu + nx and nx at
    most warp_max_nv, no slacks."""
    return (max(qp.nx[n] + qp.nu[n] for n in range(qp.N + 1)) <= warp_max_nv and max(qp.nx) <= warp_max_nv
            and all(qp.ns(n) == 0 for n in range(qp.N + 1)))


def work_split(qps, stats, warp_max_nv: int = 32):
    """Algorithmic flops of one batch solve split by arithmetic type: FP32
    (factorisations and solves with the FP32 factor), FP64 (with the FP64
    factor, and the block kernel's residuals) and double-float (the residuals
    of the one-warp kernel's FP32 iterations)."""
    f32 = f64 = fdf = 0.0
    for qp, st in zip(qps, stats):
        f, s, r = qp_flops(qp)
        nf = int(st["n_fact"])
        nf64 = int(st["n_fact64"])
        frac64 = nf64 / nf if nf else 0.0
        ns = int(st["n_solve"])
        nr = int(st["n_res"])
        f64 += nf64 * f + ns * s * frac64
        f32 += (nf - nf64) * f + ns * s * (1.0 - frac64)
        if in_warp_kernel(qp, warp_max_nv):
            fdf += nr * r * (1.0 - frac64)
            f64 += nr * r * frac64
        else:
            f64 += nr * r
    return f32, f64, fdf


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        out_dir = os.environ.get("GQ_BENCH_OUT", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle baseline
# ----------------------------------------------------------------------------
def _oracle_worker(indices):
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle import ocp_ipm as O
    from paper_2003_02547_gb300 import workloads as W
    ok = 0
    for i in indices:
        r = O.solve(W.mass_spring_qp(i, M=MASSES, N=HORIZON), O.IpmArg(tol_stat=1e-8, tol_eq=1e-8,
                                                                        tol_ineq=1e-8, tol_comp=1e-8))
        ok += r.status == O.CONVERGED
    return ok


def cpu_oracle(sample: int, offset: int = 0):
    """Solve `sample` QPs of the workload with the CPU oracle on a spawn pool
    of single-threaded workers over the host cores; returns (QP/s, cores)."""
    import multiprocessing as mp
    cores = min(os.cpu_count() or 1, 64, sample)
    env_keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        chunks = [list(range(offset + c, offset + sample, cores)) for c in range(cores)]
        with ctx.Pool(cores) as pool:
            pool.map(_oracle_worker, [[offset]] * cores)   # import + warm the workers
            t0 = time.perf_counter()
            ok = sum(pool.map(_oracle_worker, chunks))
            dt = time.perf_counter() - t0
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return sample / dt, cores, ok, dt


# ----------------------------------------------------------------------------
def launches_per_solve(qps, arg) -> int:
    """Kernel launches of one mixed gq_solve: QPs whose stages fit one warp
    run in the FP32 mirror copy, the mixed warp kernel and its FP64
    continuation launch; larger QPs in one block kernel launch."""
    warp = any(max(q.nx[n] + q.nu[n] for n in range(q.N + 1)) <= 32 and max(q.nx) <= 32 for q in qps)
    block = any(not (max(q.nx[n] + q.nu[n] for n in range(q.N + 1)) <= 32 and max(q.nx) <= 32) for q in qps)
    return (3 if arg.fp64_fallback else 2) * warp + block


# ----------------------------------------------------------------------------
# serving: open-loop Poisson arrivals through the continuous-batching server
# ----------------------------------------------------------------------------
def serving_run(rate: float, duration: float, budget_gb: float = 64.0, lanes: int = 4, max_batch: int = 512):
    """Arrivals drawn like the ragged workload (30 % repeats of an earlier key
    with x0 + N(0, 0.01^2), warm-started from the resident iterate), every
    request packed on the host before its arrival time, submitted at its
    scheduled time; latency = scheduled arrival -> solution in host memory."""
    import numpy as np
    from paper_2003_02547_gb300 import server as S, workloads as W
    from paper_2003_02547_gb300.batch import QpBatch
    arr = W.serving_arrivals(rate=rate, duration=duration, seed_pool=256)
    src = QpBatch([x.qp for x in arr], device=None)
    budget = int(budget_gb * (1 << 30))
    with S.Server(budget, lanes=lanes, max_batch=max_batch, cache_bytes=budget // 8,
                  pinned_bytes=2 << 30) as srv:
        t0 = S.now_ns() + 5_000_000
        tickets = []
        for i, x in enumerate(arr):
            due = t0 + int(x.t * 1e9)
            while S.now_ns() < due:
                pass
            tickets.append(srv.submit(src, i, key=x.key + 1, warm=x.warm, t_arrival_ns=due))
        srv.drain(600.0)
        t_end = S.now_ns()
        rep = srv.report()
        infos = [srv.result(t)[0] for t in tickets]
    lat = np.array([inf.latency_ns for inf in infos], dtype=np.float64) * 1e-6
    done_at = np.array([float(arr[i].t) * 1e3 + lat[i] for i in range(len(arr))])  # ms after t0
    in_window = int(np.sum(done_at <= duration * 1e3))
    wait = np.array([inf.wait_ns for inf in infos], dtype=np.float64) * 1e-6
    ok = np.array([inf.code == 0 and inf.stats.status == 0 for inf in infos])
    warm = np.array([bool(inf.warm_used) for inf in infos])
    iters = np.array([inf.stats.iters for inf in infos])
    done_last = max(float(arr[i].t) * 1e3 + lat[i] for i in range(len(arr)))
    return {
        "offered_qps": rate, "arrival_s": duration, "requests": len(arr),
        "throughput_qps": len(arr) / (done_last * 1e-3),
        "served_in_window_qps": in_window / duration, "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)), "admission_wait_share": float(wait.sum() / lat.sum()),
        "converged": int(ok.sum()), "warm_started": int(warm.sum()),
        "not_converged_status": sorted(int(inf.stats.status) for inf in infos if inf.code == 0 and inf.stats.status),
        # which requests did not converge: arrival index, key, warm request,
        # horizon and state size of the QP, status, iterations, flags
        "not_converged": [{"request": i, "key": int(arr[i].key), "warm": bool(arr[i].warm), "N": int(arr[i].qp.N),
                           "nx": int(max(arr[i].qp.nx)), "status": int(inf.stats.status),
                           "iters": int(inf.stats.iters), "flags": int(inf.stats.flags)}
                          for i, inf in enumerate(infos) if inf.code == 0 and inf.stats.status][:20],
        "rejected_or_failed": int(sum(inf.code != 0 for inf in infos)),
        # the same QPs solved cold by the CPU oracle: an infeasible QP fails
        # there too, an IPM failure of the served solve does not
        "not_converged_oracle": [oracle_status(arr[i].qp) for i, inf in enumerate(infos)
                                 if inf.code == 0 and inf.stats.status][:5],
        "iters_warm_mean": float(iters[warm].mean()) if warm.any() else None,
        "iters_cold_mean": float(iters[~warm].mean()),
        "iters_warm_hist": np.bincount(iters[warm], minlength=1).tolist() if warm.any() else [],
        "iters_cold_hist": np.bincount(iters[~warm], minlength=1).tolist(),
        "batches": rep["batches"], "mean_batch": rep["batched_qps"] / max(1, rep["batches"]),
        "max_lanes_busy": rep["max_lanes_busy"], "max_queue": rep["max_queue"],
        "cold_retries": rep["cold_retries"],
        "budget_gb": budget_gb, "lanes": lanes, "max_batch": max_batch,
        "wall_s": (t_end - t0) * 1e-9,
    }


def oracle_status(qp) -> dict:
    """Cold oracle solve of one QP at the exit rule of the bench."""
    from oracle import ocp_ipm as O
    r = O.solve(qp, O.IpmArg(tol_stat=1e-8, tol_eq=1e-8, tol_ineq=1e-8, tol_comp=1e-8))
    return {"status": int(r.status), "iters": int(r.iters), "res": [float(x) for x in r.res]}


def plain_serving_baseline(dev, sample: int = 48):
    """The plain per-QP FP64 GPU IPM on the serving request mix: the first
    `sample` requests of the serving arrivals, each solved alone (one solve
    call per QP, FP64 Riccati), back to back; solves/s and latency
    percentiles of the solve calls."""
    import numpy as np
    import torch
    from paper_2003_02547_gb300 import gq, workloads as W
    from paper_2003_02547_gb300.batch import QpBatch
    arr = W.serving_arrivals(rate=20000.0, duration=sample / 20000.0 + 1e-3, seed_pool=256)[:sample]
    arg = gq.default_arg(gq.MODE_SPEED, gq.PREC_FP64)
    ms, ok = [], 0
    for x in arr:
        b = QpBatch([x.qp], device=dev)
        b.upload()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.solve(arg)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        b.download()
        torch.cuda.synchronize()
        ok += int(b.all_stats()["status"][0] == 0)
    ms = np.array(ms)
    return {"value": 1e3 / ms.mean(), "unit": UNIT, "p50_ms": float(np.percentile(ms, 50)),
            "p99_ms": float(np.percentile(ms, 99)), "requests": len(arr), "converged": ok,
            "note": "cold solves, one QP per solve call; no queueing (a lower bound on its served latency)"}


def single_qp_latency(dev, precision: int, solves: int = 10000, graph: bool = False):
    """The single small QP (N=10, nx=4, nu=2) solved alone, back to back,
    one solve call at a time with its launches included: per-solve latency
    percentiles from CUDA events around each call.  With `graph`, one solve
    call is captured in a CUDA graph and each solve is a graph replay."""
    import numpy as np
    import torch
    from paper_2003_02547_gb300 import gq, workloads as W
    from paper_2003_02547_gb300.batch import QpBatch
    b = QpBatch([W.small_random_qp(0)], device=dev)
    arg = gq.default_arg(gq.MODE_SPEED, precision)
    b.upload()
    for _ in range(20):
        b.solve(arg)
    torch.cuda.synchronize()
    run = lambda: b.solve(arg)
    if graph:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            b.solve(arg)
        run = g.replay
        for _ in range(20):
            run()
        torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(solves)]
    for e0, e1 in evs:
        e0.record()
        run()
        e1.record()
    torch.cuda.synchronize()
    ms = np.array([e0.elapsed_time(e1) for e0, e1 in evs])
    b.download()
    torch.cuda.synchronize()
    st = b.all_stats()
    return {"solves": solves, "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "solves_per_s": float(1e3 / ms.mean()), "iters": int(st["iters"][0]), "converged": int(st["status"][0] == 0)}


def condensed_run(qps, block: int, dev, precision: int, reps: int = 3):
    """The batch partially condensed by `block` stages on the device
    (gq_condense_device, one kernel over the uploaded batch) and solved; the
    condensing kernel and the solve are timed separately with CUDA events,
    and the host condensing of the same batch is timed beside them."""
    import ctypes
    import numpy as np
    import torch
    from paper_2003_02547_gb300 import condense as CD, gq
    from paper_2003_02547_gb300.batch import QpBatch
    src = QpBatch(qps, device=dev)
    src.upload()
    dst = CD.condense_device(src, block, host_copy=False)
    lib = gq.load()
    nbytes = int(lib.gq_condense_ws_bytes(src.h, block))
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    cms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gq.check(lib.gq_condense_device(src.h, block, dst.h, ws.data_ptr(), nbytes, stream.cuda_stream))
        e1.record(stream)
        e1.synchronize()
        cms.append(e0.elapsed_time(e1))
    t0 = time.perf_counter()
    CD.condense(QpBatch(qps, device=None), range(len(qps)), block, device=None)
    t_host = time.perf_counter() - t0
    arg = gq.default_arg(gq.MODE_SPEED, precision)
    dst.solve(arg)
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dst.solve(arg)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    dst.download()
    torch.cuda.synchronize()
    st = dst.all_stats()
    sch = dst.schedule()
    return {"block": block, "value": len(qps) / (min(ms) * 1e-3), "unit": UNIT, "solve_ms": min(ms),
            "device_condense_ms": min(cms), "condense_share_of_solve": min(cms) / min(ms),
            "host_condense_s": t_host, "converged": int(np.sum(st["status"] == 0)),
            "iters_mean": float(np.mean(st["iters"])), "warp_qps": int(sch.warp_qps), "block_qps": int(sch.block_qps)}


def batch_run(qps, dev, precision: int, reps: int = 2, mode: int = 0, warp_max_nv=None):
    """Device-timed solves of one batch in one call (inputs resident)."""
    import numpy as np
    import torch
    from paper_2003_02547_gb300 import gq
    from paper_2003_02547_gb300.batch import QpBatch
    b = QpBatch(qps, device=dev)
    if warp_max_nv is not None:
        b.set_schedule(warp_max_nv)
    arg = gq.default_arg(mode, precision)
    b.upload()
    b.solve(arg)
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.solve(arg)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    b.download()
    torch.cuda.synchronize()
    st = b.all_stats()
    out = {"value": len(qps) / (min(ms) * 1e-3), "unit": UNIT, "ms": min(ms), "qps": len(qps),
           "converged": int(np.sum(st["status"] == 0)), "iters_mean": float(np.mean(st["iters"])),
           "fp64_fallback_qps": int(np.sum(st["flags"] & gq.FLAG_FP64_FALLBACK != 0)),
           "alu": alu_roofline(qps, st, min(ms) * 1e-3, 32 if warp_max_nv is None else warp_max_nv)}
    if mode == gq.MODE_BALANCE:
        out["array_qr_qps"] = int(np.sum(st["flags"] & gq.FLAG_ARRAY_QR != 0))
    del b
    torch.cuda.empty_cache()
    return out


# DRAM traffic of one warp_ipm_kernel<float> launch on this workload, from an
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum; summary in
# profiles/).  It is reported only while the kernel sources hash to the
# value recorded with the capture; after any change it reads null.
TRAFFIC_CAPTURE = {"sha256": "bc0520df921a686bf887f73c8b9e83b64293598920916fd9e81e5b46d21e3a38", "bytes": 5571538688}
KERNEL_SOURCES = ["gq_warp.cu", "gq_device.h", "gq_internal.h", "gq_launch.h", "gq_mma.h"]


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2003_02547_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured_traffic():
    if TRAFFIC_CAPTURE["sha256"] and TRAFFIC_CAPTURE["sha256"] == kernel_sources_sha256():
        return TRAFFIC_CAPTURE["bytes"]
    return None


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reference_arm(a):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    sample = max(4, min(a.cpu_sample, 64))
    vals = []
    cores = 1
    for k in range(a.warmup + a.steps):
        v, cores, ok, dt = cpu_oracle(sample, offset=k * sample % BATCH)
        if k >= a.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sample / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch": BATCH, "horizon": HORIZON, "nx": 16, "nu": 7,
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample} QPs of the workload per step (spawn pool, 1 thread/worker)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return reference_arm(a)
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"

    # CPU baseline first (spawn pool; no GPU state is inherited)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        v, cores, ok, dt = cpu_oracle(a.cpu_sample)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {a.cpu_sample} QPs of the workload ({dt:.1f} s wall, {ok} converged)"}

    from paper_2003_02547_gb300 import build, gq, workloads as W
    from paper_2003_02547_gb300.batch import QpBatch
    build.build()

    # one global list of world * batch QPs, split by the LPT rule on the
    # per-QP cost (every QP of this workload has the same sizes, so one cost
    # stands for all); each rank solves its shard, no data-path collective
    from paper_2003_02547_gb300 import shard
    cost = shard.qp_cost(W.mass_spring_qp(0, M=MASSES, N=HORIZON))
    mine = shard.lpt_shard([cost] * (world * a.batch), world)[rank]
    qps = [W.mass_spring_qp(i, M=MASSES, N=HORIZON) for i in mine]
    b = QpBatch(qps, device=dev)
    arg_mixed = gq.default_arg(gq.MODE_SPEED, gq.PREC_MIXED)
    arg_fp64 = gq.default_arg(gq.MODE_SPEED, gq.PREC_FP64)
    stream = torch.cuda.current_stream()
    b.upload()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2
    measure_peaks(stream.cuda_stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- device-timed batched mixed solves ----------------
    for _ in range(a.warmup):
        flush.zero_()
        b.solve(arg_mixed)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    barrier()
    for e0, e1 in evs:
        flush.zero_()                       # L2 flush between timed steps, outside the events
        e0.record(stream)
        b.solve(arg_mixed)
        e1.record(stream)
    barrier()
    ck = clocks.stop()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    launches = a.steps * launches_per_solve(qps, arg_mixed)
    b.download()
    torch.cuda.synchronize()
    st = b.all_stats()
    conv = int(np.sum(st["status"] == 0))
    fallback = int(np.sum(st["flags"] & gq.FLAG_FP64_FALLBACK != 0))
    bad = torch.tensor([a.batch - conv], device=dev, dtype=torch.int64)
    if world > 1:
        dist.all_reduce(bad)       # every rank leaves together when any rank failed
    if int(bad.item()) != 0:
        # a timed run with an unconverged QP is a failed run, not a number
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": None, "unit": UNIT, "n_gpus": world,
                              "error": f"{int(bad.item())} QPs did not converge in the timed solves",
                              "statuses": np.bincount(st["status"], minlength=5).tolist()}), flush=True)
        return 1
    mean_ms = statistics.mean(step_ms)
    tmax = torch.tensor([mean_ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    mean_ms_max = float(tmax.item())
    value = world * a.batch / (mean_ms_max * 1e-3)
    step_sorted = sorted(step_ms)
    p50 = float(np.percentile(step_sorted, 50))
    p99 = float(np.percentile(step_sorted, 99))

    # ---------------- roofline of the IPM kernel ----------------
    f32, f64, fdf = work_split(qps, st)
    t_kernel = mean_ms * 1e-3
    t_min = t_min_of(f32, f64, fdf)
    achieved = (f32 + f64 + fdf) / t_kernel
    peak_eff = (f32 + f64 + fdf) / t_min if t_min > 0 else float("nan")
    # the same flops with the residual mat-vecs counted at the FP64 rate (the
    # bound of an FP64 residual, the precision they stand in for)
    t_min64 = f32 / PEAKS["fp32"] + (f64 + fdf) / PEAKS["fp64"]

    # ---------------- e2e through the C ABI with host buffers ----------------
    for _ in range(2):
        b.upload()
        b.solve(arg_mixed)
        b.download()
    barrier()
    e2e_ms = []
    for _ in range(max(3, a.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.upload()
        b.solve(arg_mixed)
        b.download()
        stream.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    st_e2e = b.all_stats()
    e2e_ok = int(np.sum(st_e2e["status"] == 0))
    bad = torch.tensor([a.batch - e2e_ok], device=dev, dtype=torch.int64)
    if world > 1:
        dist.all_reduce(bad)
    if int(bad.item()) != 0:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": None, "unit": UNIT, "n_gpus": world,
                              "error": f"{int(bad.item())} QPs did not converge in the e2e solves"}),
                  flush=True)
        return 1
    e2e_val = a.batch / (statistics.mean(e2e_ms) * 1e-3)

    # ---------------- batched FP64 and plain per-QP FP64 GPU baselines ----------------
    for _ in range(2):
        b.solve(arg_fp64)
    barrier()
    f64_ms = []
    for _ in range(3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.solve(arg_fp64)
        e1.record(stream)
        e1.synchronize()
        f64_ms.append(e0.elapsed_time(e1))
    b.download()
    torch.cuda.synchronize()
    st64 = b.all_stats()
    batched_fp64 = a.batch / (statistics.mean(f64_ms) * 1e-3)
    plain_ms = []
    plain_ok = 0
    singles = [QpBatch([q], device=dev) for q in qps[:a.plain_sample]]
    for sb in singles:
        sb.upload()
        sb.solve(arg_fp64)
    torch.cuda.synchronize()
    for sb in singles:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sb.solve(arg_fp64)
        e1.record(stream)
        e1.synchronize()
        plain_ms.append(e0.elapsed_time(e1))
        sb.download()
        torch.cuda.synchronize()
        plain_ok += int(sb.all_stats()["status"][0] == 0)
    plain = {"value": 1e3 / statistics.mean(plain_ms), "unit": UNIT,
             "p50_ms": float(np.percentile(plain_ms, 50)), "p99_ms": float(np.percentile(plain_ms, 99)),
             "sample": f"{a.plain_sample} QPs, one launch each, FP64 Riccati", "converged": plain_ok}

    extras = {}
    if rank == 0 and world == 1 and not a.no_extras:
        del singles
        extras["mass_spring_condensed_2_mixed"] = condensed_run(qps, 2, dev, gq.PREC_MIXED)
        # the solver modes of Sec. 4.2 on the same batch (the paper compares
        # speed and robust on this model): time per solve relative to speed
        modes = {}
        for name, mode, prec in (("speed_fp64", gq.MODE_SPEED, gq.PREC_FP64),
                                 ("balance_fp64", gq.MODE_BALANCE, gq.PREC_FP64),
                                 ("robust_fp64", gq.MODE_ROBUST, gq.PREC_FP64),
                                 ("speed_mixed", gq.MODE_SPEED, gq.PREC_MIXED),
                                 ("robust_mixed", gq.MODE_ROBUST, gq.PREC_MIXED)):
            modes[name] = batch_run(qps, dev, prec, mode=mode)
        for name in ("balance_fp64", "robust_fp64"):
            modes[name]["time_vs_speed"] = modes[name]["ms"] / modes["speed_fp64"]["ms"]
        modes["robust_mixed"]["time_vs_speed"] = modes["robust_mixed"]["ms"] / modes["speed_mixed"]["ms"]
        extras["mass_spring_modes"] = modes
        extras["single_small_qp_mixed"] = single_qp_latency(dev, gq.PREC_MIXED)
        extras["single_small_qp_fp64"] = single_qp_latency(dev, gq.PREC_FP64)
        extras["single_small_qp_mixed_graph"] = single_qp_latency(dev, gq.PREC_MIXED, graph=True)
        ragged = W.ragged_batch(4096)
        extras["ragged_4096_mixed"] = batch_run(ragged, dev, gq.PREC_MIXED)
        extras["ragged_4096_fp64"] = batch_run(ragged, dev, gq.PREC_FP64)
        del ragged
        large = W.large_stage_batch(256)
        extras["large_stage_256_mixed"] = batch_run(large, dev, gq.PREC_MIXED, reps=1)
        extras["large_stage_256_fp64"] = batch_run(large, dev, gq.PREC_FP64, reps=1)
        del large
        extras["serving"] = serving_run(a.serving_rate, a.serving_duration)
        # offered-load sweep over the same request mix: the sustained rate is
        # the largest offered load the server keeps up with (served rate over
        # the arrival window at least 90 % of the offered one); latency there
        # is without a standing queue
        sweep = []
        for rate in (100.0, 200.0, 400.0):
            r = serving_run(rate, 2.0)
            r["sustained"] = bool(r["served_in_window_qps"] >= 0.9 * rate)
            sweep.append(r)
        extras["serving_sweep"] = sweep
        # the same 400 QP/s load with 16 lanes (micro-batches in flight)
        r16 = serving_run(400.0, 2.0, lanes=16)
        r16["sustained"] = bool(r16["served_in_window_qps"] >= 0.9 * 400.0)
        extras["serving_400_lanes16"] = r16
        ok = [r for r in sweep if r["sustained"]]
        extras["serving_sustained_qps"] = max((r["offered_qps"] for r in ok), default=None)
        extras["serving_plain_fp64_gpu"] = plain_serving_baseline(dev, sample=48)
        # soft constraints (Sec. 2.2): every state box of the mass-spring batch
        # soft (L2 + L1 penalty); QPs with slacks run in the block kernel, so
        # the hard batch is timed there too.  Reported, not fatal to the line.
        try:
            soft = [W.soften(q, range(1, q.N + 1), "x", Z=10.0, z=1.0, ls=0.0) for q in qps]
            extras["mass_spring_soft_states"] = {
                "slack_pairs_per_qp": int(sum(soft[0].ns(n) for n in range(soft[0].N + 1))),
                "soft_mixed": batch_run(soft, dev, gq.PREC_MIXED),
                "soft_fp64": batch_run(soft, dev, gq.PREC_FP64),
                "hard_block_kernel_mixed": batch_run(qps, dev, gq.PREC_MIXED, warp_max_nv=0),
                "hard_block_kernel_fp64": batch_run(qps, dev, gq.PREC_FP64, warp_max_nv=0)}
        except Exception as e:
            extras["mass_spring_soft_states"] = {"error": repr(e)[:300]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": mean_ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch_per_gpu": a.batch, "horizon": HORIZON, "nx": 16, "nu": 7,
                       "precision": "mixed (FP32 Riccati, FP64 residual/IR/step)", "kkt_tol": 1e-8,
                       "l2": "flushed between timed steps (256 MB write)"},
            "p50_ms": p50, "p99_ms": p99,
            "converged": conv, "fp64_fallback_qps": fallback,
            "iters_mean": float(np.mean(st["iters"])), "ir_mean": float(np.mean(st["ir_total"])),
            "gpu_launches": launches,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_eff / 1e12, "unit": "TFLOP/s",
                         "frac": achieved / peak_eff if peak_eff == peak_eff else None, "traffic": captured_traffic(),
                         "kernel": "warp_ipm_kernel<float>", "flops_f32": f32, "flops_f64": f64,
                         "flops_df": fdf,
                         "peak_fp32_tflops": PEAKS["fp32"] / 1e12, "peak_fp64_tflops": PEAKS["fp64"] / 1e12,
                         "frac_residuals_at_fp64_rate": t_min64 / t_kernel,
                         "peak_note": f"FP32 and FP64 FMA peaks {PEAKS['source']} (nominal 80.5 and 1.25 TF); "
                                      f"peak = flop-mix-weighted, each class on the unit that runs it (double-float "
                                      f"residual mat-vecs at 1/{DF_COST:g} of the FP32 rate)"},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(b.sizes.in_bytes),
                    "d2h_bytes_per_step": int(b.sizes.sol_bytes), "converged": e2e_ok},
            "batched_fp64_gpu": {"value": batched_fp64, "unit": UNIT, "ms": statistics.mean(f64_ms),
                                 "converged": int(np.sum(st64["status"] == 0)),
                                 "iters_mean": float(np.mean(st64["iters"]))},
            "plain_fp64_gpu": plain,
            "clocks": ck,
            "cpu_baseline": cpu,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
