"""ctypes binding of libgq, the C ABI declared in include/gq.h.

Argument marshalling only: every step of the solver runs in the CUDA library.
Importing this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgq.so")

GQ_OK = 0
GQ_ERR_ARG, GQ_ERR_DIMS, GQ_ERR_SIZE, GQ_ERR_CUDA, GQ_ERR_DATA, GQ_ERR_STATE = -1, -2, -3, -4, -5, -6
STATUS_CONVERGED, STATUS_MAX_ITER, STATUS_MIN_STEP, STATUS_NAN, STATUS_TIMEOUT = 0, 1, 2, 3, 4
FLAG_FP64_FALLBACK = 1
FLAG_REGULARIZED = 2
FLAG_ARRAY_QR = 4
MODE_SPEED, MODE_BALANCE, MODE_ROBUST = 0, 1, 2
PREC_FP64, PREC_MIXED = 0, 1

c_int, c_int64, c_double, c_size_t, c_void_p = (ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                                ctypes.c_size_t, ctypes.c_void_p)
P_int = ctypes.POINTER(ctypes.c_int)
P_double = ctypes.POINTER(ctypes.c_double)


class IpmArg(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("precision", ctypes.c_int32), ("iter_max", ctypes.c_int32),
                ("warm_start", ctypes.c_int32), ("ir_steps", ctypes.c_int32), ("cond_corr", ctypes.c_int32),
                ("fp64_fallback", ctypes.c_int32), ("riccati", ctypes.c_int32),
                ("tol_stat", c_double), ("tol_eq", c_double), ("tol_ineq", c_double), ("tol_comp", c_double),
                ("alpha_min", c_double), ("lam_min", c_double), ("t_min", c_double), ("tau_b", c_double),
                ("corr_k", c_double), ("reg_prim", c_double), ("ir_tol", c_double), ("warm_min", c_double),
                ("timeout_ns", c_int64), ("ir_fail_ratio", c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("ir_total", ctypes.c_int32), ("n_fact", ctypes.c_int32), ("n_fact64", ctypes.c_int32),
                ("n_solve", ctypes.c_int32), ("n_res", ctypes.c_int32), ("res", c_double * 4)]


class Sizes(ctypes.Structure):
    _fields_ = [("in_bytes", c_size_t), ("sol_bytes", c_size_t), ("ws_bytes", c_size_t),
                ("n_stages", c_int64), ("n_slots", c_int64), ("nv_total", c_int64),
                ("neq_total", c_int64), ("nside_total", c_int64), ("nv_max", ctypes.c_int32),
                ("nx_max", ctypes.c_int32)]


class Schedule(ctypes.Structure):
    _fields_ = [("warp_max_nv", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("warp_qps", ctypes.c_int32), ("block_qps", ctypes.c_int32), ("tensor_cores", ctypes.c_int32)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("max_wait_us", ctypes.c_int32),
                ("device", ctypes.c_int32), ("cache_bytes", c_size_t), ("arg", IpmArg),
                ("class_ratio", c_double)]


class Request(ctypes.Structure):
    _fields_ = [("src", c_void_p), ("src_qp", ctypes.c_int32), ("warm", ctypes.c_int32),
                ("key", ctypes.c_uint64), ("t_arrival_ns", c_int64),
                ("y", P_double), ("pi", P_double), ("lam", P_double), ("t", P_double)]


class TicketInfo(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("code", ctypes.c_int32), ("warm_used", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("latency_ns", c_int64), ("wait_ns", c_int64),
                ("stats", Stats)]


class ServerReport(ctypes.Structure):
    _fields_ = [(n, c_int64) for n in ("submitted", "completed", "rejected", "failed", "batches", "batched_qps",
                                       "warm_hits", "warm_misses", "cache_entries", "cache_evictions",
                                       "cache_skips", "deferrals", "max_lanes_busy", "max_queue", "cold_retries")]


# name -> (restype, argtypes); the same names and order as include/gq.h and
# include/gq_server.h
SIGNATURES = {
    "gq_ipm_arg_default": (c_int, [ctypes.POINTER(IpmArg), c_int, c_int]),
    "gq_batch_memsize": (c_size_t, [c_int, P_int, c_size_t, P_int]),
    "gq_batch_create": (c_int, [c_int, P_int, c_size_t, P_int, c_void_p, c_size_t, ctypes.POINTER(c_void_p)]),
    "gq_batch_create_soft": (c_int, [c_int, P_int, c_size_t, P_int, P_int, c_void_p, c_size_t,
                                     ctypes.POINTER(c_void_p)]),
    "gq_batch_sizes": (c_int, [c_void_p, ctypes.POINTER(Sizes)]),
    "gq_batch_attach": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "gq_set_dynamics": (c_int, [c_void_p, c_int, c_int, P_double, c_int, P_double, c_int, P_double]),
    "gq_set_cost": (c_int, [c_void_p, c_int, c_int, P_double, c_int, P_double, c_int, P_double, c_int,
                            P_double, P_double]),
    "gq_set_box": (c_int, [c_void_p, c_int, c_int, P_int, P_double, P_double, P_int, P_double, P_double]),
    "gq_set_general": (c_int, [c_void_p, c_int, c_int, P_double, c_int, P_double, c_int, P_double, P_double]),
    "gq_set_soft": (c_int, [c_void_p, c_int, c_int, P_int, P_double, P_double, P_double, P_double, P_double,
                            P_double]),
    "gq_set_guess": (c_int, [c_void_p, c_int, P_double, P_double, P_double, P_double]),
    "gq_get_dynamics": (c_int, [c_void_p, c_int, c_int, P_double, c_int, P_double, c_int, P_double]),
    "gq_get_cost": (c_int, [c_void_p, c_int, c_int, P_double, c_int, P_double, c_int, P_double, c_int,
                            P_double, P_double]),
    "gq_get_box": (c_int, [c_void_p, c_int, c_int, P_int, P_double, P_double, P_int, P_double, P_double]),
    "gq_get_general": (c_int, [c_void_p, c_int, c_int, P_double, c_int, P_double, c_int, P_double, P_double]),
    "gq_get_soft": (c_int, [c_void_p, c_int, c_int, P_int, P_int, P_double, P_double, P_double, P_double, P_double,
                            P_double]),
    "gq_condense_dims": (c_int, [c_void_p, c_int, c_int, P_int, c_size_t, ctypes.POINTER(c_size_t)]),
    "gq_condense": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int]),
    "gq_expand": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, P_double, P_double, P_double, P_double,
                          P_double, P_double, P_double, P_double]),
    "gq_condense_ws_bytes": (c_size_t, [c_void_p, c_int]),
    "gq_condense_device": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gq_set_initial_state": (c_int, [c_void_p, c_int, P_double, c_int, P_double, c_int, P_double, P_double, c_int,
                                     P_double, P_double, c_int, P_double, P_double]),
    "gq_copy_qp": (c_int, [c_void_p, c_int, c_void_p, c_int]),
    "gq_get_schedule": (c_int, [c_void_p, ctypes.POINTER(Schedule)]),
    "gq_set_schedule": (c_int, [c_void_p, ctypes.POINTER(Schedule)]),
    "gq_autotune": (c_int, [c_void_p, ctypes.POINTER(IpmArg), c_void_p, c_int, ctypes.POINTER(Schedule),
                            ctypes.POINTER(c_double)]),
    "gq_upload": (c_int, [c_void_p, c_void_p]),
    "gq_upload_sol": (c_int, [c_void_p, c_void_p]),
    "gq_download": (c_int, [c_void_p, c_void_p]),
    "gq_solve": (c_int, [c_void_p, ctypes.POINTER(IpmArg), c_void_p]),
    "gq_residuals": (c_int, [c_void_p, c_void_p]),
    "gq_newton_step": (c_int, [c_void_p, ctypes.POINTER(IpmArg), c_double, c_void_p, c_void_p]),
    "gq_noalloc_scratch_bytes": (c_size_t, []),
    "gq_solve_noalloc": (c_int, [c_void_p, ctypes.POINTER(IpmArg), c_void_p, c_void_p, c_void_p]),
    "gq_get_stage_sol": (c_int, [c_void_p, c_int, c_int, P_double, P_double, P_double, P_double, P_double]),
    "gq_get_stage_slacks": (c_int, [c_void_p, c_int, c_int, P_double, P_double]),
    "gq_get_stats": (c_int, [c_void_p, c_int, ctypes.POINTER(Stats)]),
    "gq_get_statuses": (c_int, [c_void_p, P_int, P_int]),
    "gq_get_sol_offsets": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int64)]),
    "gq_probe_fma_rate": (c_int, [c_int, c_void_p, P_double]),
    "gq_last_error": (ctypes.c_char_p, []),
    "gq_server_cfg_default": (c_int, [ctypes.POINTER(ServerCfg)]),
    "gq_server_create": (c_int, [ctypes.POINTER(ServerCfg), c_void_p, c_size_t, c_void_p, c_size_t,
                                 ctypes.POINTER(c_void_p)]),
    "gq_server_submit": (c_int, [c_void_p, ctypes.POINTER(Request), ctypes.POINTER(c_int64)]),
    "gq_server_poll": (c_int, [c_void_p, c_int64, ctypes.POINTER(TicketInfo)]),
    "gq_server_drain": (c_int, [c_void_p, c_int64]),
    "gq_server_report_get": (c_int, [c_void_p, ctypes.POINTER(ServerReport)]),
    "gq_server_destroy": (c_int, [c_void_p]),
}

_lib = None


def load():
    """Load libgq.so (built by paper_2003_02547_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgq.so not built at {LIB_PATH}: run paper_2003_02547_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GqError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gq error {code}: {msg}")
        self.code = code


def check(rc: int) -> int:
    if rc != GQ_OK:
        raise GqError(rc, load().gq_last_error().decode())
    return rc


def _bind(name):
    def call(*args):
        return getattr(load(), name)(*args)
    call.__name__ = name
    call.__doc__ = f"libgq {name} (see include/gq.h)"
    return call


# module-level functions with the C names
for _n in SIGNATURES:
    globals()[_n] = _bind(_n)


def noalloc_scratch_bytes() -> int:
    """Bytes of the static workspace of gq_solve_noalloc, as compiled into the library."""
    return int(load().gq_noalloc_scratch_bytes())


def default_arg(mode: int = MODE_SPEED, precision: int = PREC_FP64, **over) -> IpmArg:
    a = IpmArg()
    check(load().gq_ipm_arg_default(ctypes.byref(a), mode, precision))
    for k, v in over.items():
        if not hasattr(a, k):
            raise AttributeError(k)
        setattr(a, k, v)
    return a
