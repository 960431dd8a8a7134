"""The C ABI on the host: the library loads, exports every declared symbol,
and its planner and setters validate input.  No GPU call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gqmod():
    from paper_2003_02547_gb300 import build
    build.build()
    from paper_2003_02547_gb300 import gq
    gq.load()
    return gq


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"GQ_API\s+[\w\s\*]+?\b(gq_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gq_batch_create", "gq_solve", "gq_set_dynamics", "gq_get_stage_sol", "gq_newton_step"):
        assert must in names


def test_library_exports_every_declared_symbol(gqmod):
    lib = gqmod.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in gqmod.SIGNATURES, f"binding lacks {name}"


def test_binding_names_match_header(gqmod):
    assert sorted(gqmod.SIGNATURES) == declared_functions()


def test_struct_sizes_match_header(gqmod):
    assert ctypes.sizeof(gqmod.IpmArg) == 8 * 4 + 12 * 8 + 8 + 8
    assert ctypes.sizeof(gqmod.Stats) == 64
    assert ctypes.sizeof(gqmod.ServerCfg) == 4 * 4 + 8 + ctypes.sizeof(gqmod.IpmArg) + 8
    assert ctypes.sizeof(gqmod.Request) == 8 + 4 + 4 + 8 + 8 + 4 * 8
    assert ctypes.sizeof(gqmod.TicketInfo) == 4 * 4 + 2 * 8 + 64
    assert ctypes.sizeof(gqmod.ServerReport) == 15 * 8


def test_noalloc_scratch_size_matches_header(gqmod):
    src = open(os.path.join(ROOT, "include", "gq.h")).read()
    m = re.search(r"#define GQ_NOALLOC_SCRATCH_BYTES \((\d+)u \* 1024u \* 1024u\)", src)
    assert m, "GQ_NOALLOC_SCRATCH_BYTES not found in gq.h"
    assert gqmod.noalloc_scratch_bytes() == int(m.group(1)) * 1024 * 1024


def test_arg_defaults(gqmod):
    a = gqmod.default_arg(gqmod.MODE_SPEED, gqmod.PREC_FP64)
    assert a.tol_stat == 1e-8 and a.tau_b == 0.995 and a.ir_steps == 0 and a.reg_prim == 0.0
    m = gqmod.default_arg(gqmod.MODE_SPEED, gqmod.PREC_MIXED)
    assert m.ir_steps == 3 and m.reg_prim > 0
    bad = gqmod.IpmArg()
    assert gqmod.load().gq_ipm_arg_default(ctypes.byref(bad), 7, 0) == gqmod.GQ_ERR_ARG
    assert "mode" in gqmod.load().gq_last_error().decode()


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def test_memsize_rejects_bad_dims(gqmod):
    lib = gqmod.load()
    for dims in ([2, 1, 1, 0, 0, 0], [0, -1, 1, 0, 0, 0], [0, 1, 1, 2, 0, 0], [0, 0, 0, 0, 0, 0]):
        d, p = _i(dims)
        assert lib.gq_batch_memsize(1, p, d.size, None) == 0
    d, p = _i([0, 1, 1, 0, 0, 0])
    assert lib.gq_batch_memsize(1, p, d.size, None) > 0


def test_layout_and_slot_sharing(gqmod):
    from paper_2003_02547_gb300 import workloads as W
    from paper_2003_02547_gb300.batch import QpBatch
    qps = [W.mass_spring_qp(i) for i in range(8)]
    shared = QpBatch(qps, device=None, share=True)
    private = QpBatch(qps, device=None, share=False)
    assert shared.sizes.n_stages == private.sizes.n_stages == 8 * 31
    assert shared.sizes.n_slots == 8 + 2          # stage 0 per QP, middle and terminal shared
    assert private.sizes.n_slots == 8 * 31
    assert shared.sizes.in_bytes < private.sizes.in_bytes
    assert shared.sizes.nv_total == 8 * (7 + 29 * 23 + 16)
    assert shared.sizes.nv_max == 23 and shared.sizes.nx_max == 16
    o = shared.offsets(3)
    assert o[4] == 7 + 29 * 23 + 16 and o[5] == 30 * 16 and o[6] == 2 * (7 + 29 * 23 + 16)


def test_slot_with_mismatched_sizes_is_rejected(gqmod):
    lib = gqmod.load()
    d, dp = _i([1, 2, 1, 0, 0, 0, 2, 0, 0, 0, 0])   # N=1: stage0 (2,1), stage1 (2,0)
    s, sp = _i([5, 5])
    mem = lib.gq_batch_memsize(1, dp, d.size, sp)
    buf = np.zeros(mem + 64, dtype=np.uint8)
    ptr = buf.ctypes.data + (-buf.ctypes.data) % 64
    h = ctypes.c_void_p()
    assert lib.gq_batch_create(1, dp, d.size, sp, ptr, mem, ctypes.byref(h)) == gqmod.GQ_ERR_DIMS


def test_setters_validate(gqmod):
    from paper_2003_02547_gb300 import workloads as W
    from paper_2003_02547_gb300.batch import QpBatch, _ptr, _f64
    b = QpBatch([W.small_random_qp(0)], device=None)
    lib, h = b.lib, b.h
    D = ctypes.POINTER(ctypes.c_double)
    # stage out of range, qp out of range
    A = _f64(np.eye(4))
    B = _f64(np.ones((4, 2)))
    bb = _f64(np.zeros(4))
    assert lib.gq_set_dynamics(h, 0, 99, _ptr(A), 4, _ptr(B), 4, _ptr(bb)) == gqmod.GQ_ERR_ARG
    assert lib.gq_set_dynamics(h, 5, 1, _ptr(A), 4, _ptr(B), 4, _ptr(bb)) == gqmod.GQ_ERR_ARG
    # terminal stage has no dynamics
    assert lib.gq_set_dynamics(h, 0, 10, _ptr(A), 4, _ptr(B), 4, _ptr(bb)) == gqmod.GQ_ERR_ARG
    # leading dimension too small
    assert lib.gq_set_dynamics(h, 0, 1, _ptr(A), 2, _ptr(B), 4, _ptr(bb)) == gqmod.GQ_ERR_ARG
    # NaN data
    An = _f64(np.eye(4))
    An[1, 2] = np.nan
    assert lib.gq_set_dynamics(h, 0, 1, _ptr(An), 4, _ptr(B), 4, _ptr(bb)) == gqmod.GQ_ERR_DATA
    # non-symmetric Q
    Q = _f64(np.eye(4))
    Q[0, 1] = 1.0
    S = _f64(np.zeros((2, 4)))
    R = _f64(np.eye(2))
    q = _f64(np.zeros(4))
    r = _f64(np.zeros(2))
    assert lib.gq_set_cost(h, 0, 1, _ptr(Q), 4, _ptr(S), 2, _ptr(R), 2, _ptr(q), _ptr(r)) == gqmod.GQ_ERR_DATA
    # box: index out of range, repeated index, lo > hi
    iu, ip = _i([0, 5])
    lb = _f64([-1, -1])
    ub = _f64([1, 1])
    ix, xp = _i([0, 1, 2, 3])
    lx = _f64([-5] * 4)
    ux = _f64([5] * 4)
    assert lib.gq_set_box(h, 0, 1, ip, _ptr(lb), _ptr(ub), xp, _ptr(lx), _ptr(ux)) == gqmod.GQ_ERR_ARG
    iu, ip = _i([1, 1])
    assert lib.gq_set_box(h, 0, 1, ip, _ptr(lb), _ptr(ub), xp, _ptr(lx), _ptr(ux)) == gqmod.GQ_ERR_ARG
    iu, ip = _i([0, 1])
    assert lib.gq_set_box(h, 0, 1, ip, _ptr(_f64([2, -1])), _ptr(ub), xp, _ptr(lx), _ptr(ux)) == gqmod.GQ_ERR_DATA
    assert lib.gq_set_box(h, 0, 1, ip, _ptr(lb), _ptr(ub), xp, _ptr(lx), _ptr(ux)) == gqmod.GQ_OK
    # infinite bounds mask a side and are accepted
    assert lib.gq_set_box(h, 0, 1, ip, _ptr(_f64([-np.inf, -1])), _ptr(_f64([1, np.inf])), xp, _ptr(lx),
                          _ptr(ux)) == gqmod.GQ_OK
    assert lib.gq_set_box(h, 0, 1, ip, _ptr(_f64([np.inf, -1])), _ptr(ub), xp, _ptr(lx),
                          _ptr(ux)) == gqmod.GQ_ERR_DATA
    del D


def test_solve_rejects_bad_arguments_before_launch(gqmod):
    from paper_2003_02547_gb300 import workloads as W
    from paper_2003_02547_gb300.batch import QpBatch
    b = QpBatch([W.small_random_qp(0)], device=None)
    lib = b.lib
    for field, val in (("tau_b", 1.5), ("lam_min", 0.0), ("warm_start", 3), ("iter_max", -1),
                       ("precision", 9), ("timeout_ns", -5)):
        a = gqmod.default_arg()
        setattr(a, field, val)
        assert lib.gq_solve(b.h, ctypes.byref(a), None) == gqmod.GQ_ERR_ARG, field


def test_guess_and_offsets_roundtrip_on_host(gqmod):
    from paper_2003_02547_gb300 import workloads as W
    from paper_2003_02547_gb300.batch import QpBatch
    qps = [W.small_random_qp(i) for i in range(3)]
    b = QpBatch(qps, device=None)
    o = b.offsets(1)
    y = np.arange(o[4], dtype=np.float64)
    lam = np.linspace(0, 1, o[6])
    b.set_guess(1, y=y, lam=lam)
    yy, pp, ll, tt = b.solution(1)
    np.testing.assert_array_equal(yy, y)
    np.testing.assert_array_equal(ll, lam)


def test_server_create_validates_before_any_cuda_call(gqmod):
    lib = gqmod.load()
    cfg = gqmod.ServerCfg()
    assert lib.gq_server_cfg_default(ctypes.byref(cfg)) == 0
    assert cfg.lanes == 4 and cfg.max_batch == 256 and cfg.arg.precision == gqmod.PREC_MIXED
    assert cfg.class_ratio == 4.0
    out = ctypes.c_void_p()
    buf = np.zeros(1 << 16, dtype=np.uint8)
    base = buf.ctypes.data + ((-buf.ctypes.data) % 256)
    assert lib.gq_server_create(None, base, 4096, base, 4096, ctypes.byref(out)) == gqmod.GQ_ERR_ARG
    bad = gqmod.ServerCfg()
    lib.gq_server_cfg_default(ctypes.byref(bad))
    bad.lanes = 0
    assert lib.gq_server_create(ctypes.byref(bad), base, 4096, base, 4096, ctypes.byref(out)) == gqmod.GQ_ERR_ARG
    assert "lanes" in lib.gq_last_error().decode()
    bad.lanes = 2
    assert lib.gq_server_create(ctypes.byref(bad), base + 8, 4096, base, 4096, ctypes.byref(out)) == gqmod.GQ_ERR_ARG
    bad.cache_bytes = 1 << 20  # cache larger than the arena
    assert lib.gq_server_create(ctypes.byref(bad), base, 4096, base, 4096, ctypes.byref(out)) == gqmod.GQ_ERR_SIZE
    assert out.value is None
    info = gqmod.TicketInfo()
    assert lib.gq_server_poll(None, 0, ctypes.byref(info)) == gqmod.GQ_ERR_ARG
    assert lib.gq_server_submit(None, None, None) == gqmod.GQ_ERR_ARG
    assert lib.gq_server_destroy(None) == gqmod.GQ_ERR_ARG


def _f(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def test_set_initial_state_folds_x0_like_the_elimination(gqmod):
    """gq_set_initial_state writes the same stage-0 data as eliminating x_0
    by hand (b_0 = b + A x0, r_0 = r + S x0, general bounds minus C x0), and
    re-applying it with another x0 gives the data of that x0."""
    from paper_2003_02547_gb300 import workloads as W
    from paper_2003_02547_gb300.batch import QpBatch
    lib = gqmod.load()
    P = ctypes.POINTER(ctypes.c_double)
    qp = W.ragged_random_qp(3)
    assert qp.ng(0) > 0
    x_new = qp.x0 + 0.05
    for x in (qp.x0, x_new):
        ref = QpBatch([W.perturb_x0(qp, x) if x is x_new else qp], device=None)
        got = QpBatch([qp], device=None)
        A, S, C = _f(qp.A[1]), _f(qp.S_full), _f(qp.C0_full)
        b0 = np.ascontiguousarray(qp.b[0] - qp.A[1] @ qp.x0)
        r0 = np.ascontiguousarray(qp.r[0] - qp.S_full @ qp.x0)
        lg0 = np.ascontiguousarray(qp.lg[0] + qp.C0_full @ qp.x0)
        ug0 = np.ascontiguousarray(qp.ug[0] + qp.C0_full @ qp.x0)
        xx = np.ascontiguousarray(x, dtype=np.float64)
        rc = lib.gq_set_initial_state(got.h, 0, xx.ctypes.data_as(P), xx.size, A.ctypes.data_as(P), A.shape[0],
                                      b0.ctypes.data_as(P), S.ctypes.data_as(P), S.shape[0], r0.ctypes.data_as(P),
                                      C.ctypes.data_as(P), C.shape[0], lg0.ctypes.data_as(P), ug0.ctypes.data_as(P))
        assert rc == 0, lib.gq_last_error().decode()
        n = got.sizes.in_bytes // 8
        a = got.host_in.view(np.float64, 0, n)
        c = ref.host_in.view(np.float64, 0, n)
        np.testing.assert_allclose(a, c, rtol=1e-13, atol=1e-13, equal_nan=True)
    b = QpBatch([qp], device=None)
    assert lib.gq_set_initial_state(b.h, 0, None, -1, None, 1, None, None, 1, None, None, 1, None, None) == \
        gqmod.GQ_ERR_ARG


def test_get_statuses_reads_every_qp(gqmod):
    from paper_2003_02547_gb300 import workloads as W
    from paper_2003_02547_gb300.batch import QpBatch
    b = QpBatch([W.small_random_qp(i) for i in range(3)], device=None)
    st = b.host_sol.view(np.int32, 0, 3 * 16)
    for q in range(3):
        st[16 * q] = q          # status
        st[16 * q + 1] = 10 + q  # iters
    out, it = np.full(3, -9, dtype=np.int32), np.full(3, -9, dtype=np.int32)
    P = ctypes.POINTER(ctypes.c_int)
    assert gqmod.load().gq_get_statuses(b.h, out.ctypes.data_as(P), it.ctypes.data_as(P)) == 0
    assert out.tolist() == [0, 1, 2] and it.tolist() == [10, 11, 12]


def test_schedule_replans_buckets(gqmod):
    from paper_2003_02547_gb300 import workloads as W
    from paper_2003_02547_gb300.batch import QpBatch
    qps = [W.small_random_qp(0), W.ragged_random_qp(0), W.mass_spring_qp(0)]
    b = QpBatch(qps, device=None)
    sch = b.schedule()
    assert (sch.warp_max_nv, sch.block_threads) == (32, 0)
    nw = sum(max(q.nx[n] + q.nu[n] for n in range(q.N + 1)) <= 32 and max(q.nx) <= 32 for q in qps)
    assert (sch.warp_qps, sch.block_qps) == (nw, len(qps) - nw)
    b.set_schedule(0, 128)
    sch = b.schedule()
    assert (sch.warp_qps, sch.block_qps, sch.block_threads) == (0, 3, 128)
    lib = gqmod.load()
    bad = gqmod.Schedule(33, 256, 0, 0)
    assert lib.gq_set_schedule(b.h, ctypes.byref(bad)) == gqmod.GQ_ERR_ARG
    bad = gqmod.Schedule(32, 96, 0, 0)
    assert lib.gq_set_schedule(b.h, ctypes.byref(bad)) == gqmod.GQ_ERR_ARG



def test_copy_qp_moves_stage_data_between_batches(gqmod):
    """gq_copy_qp copies every stage block of a QP into another batch's QP of
    the same sizes; other sizes are refused with GQ_ERR_DIMS."""
    from paper_2003_02547_gb300 import workloads as W
    from paper_2003_02547_gb300.batch import QpBatch
    lib = gqmod.load()
    src = QpBatch([W.small_random_qp(4), W.ragged_random_qp(2)], device=None)
    dst = QpBatch([W.ragged_random_qp(2), W.small_random_qp(9)], device=None, set_data=False)
    assert lib.gq_copy_qp(dst.h, 0, src.h, 1) == 0
    assert lib.gq_copy_qp(dst.h, 1, src.h, 0) == 0
    ref = QpBatch([W.ragged_random_qp(2), W.small_random_qp(4)], device=None)
    n = ref.sizes.in_bytes // 8
    np.testing.assert_array_equal(dst.host_in.view(np.uint8, 0, n * 8), ref.host_in.view(np.uint8, 0, n * 8))
    assert lib.gq_copy_qp(dst.h, 0, src.h, 0) == gqmod.GQ_ERR_DIMS
