"""Soft constraints (Sec. 2.2) in the batch layout and the C ABI, host side
(no GPU): vector lengths, the staged slack data read back through the
getters, scheduling into the block kernel, and argument validation."""
import ctypes

import numpy as np
import pytest

from oracle import ocp_ipm as O
from paper_2003_02547_gb300 import workloads as W


@pytest.fixture(scope="module")
def gqmod():
    from paper_2003_02547_gb300 import build
    build.build()
    from paper_2003_02547_gb300 import gq
    return gq


def soft_qp(seed=0):
    qp = W.small_random_qp(seed)
    return W.soften(qp, [1, 3, qp.N], "x", Z=2.0, z=0.5, ls=-0.1)


def test_layout_lengths_follow_the_oracle(gqmod):
    """y holds [u; x; s^l; s^u] per stage and lambda/t 2 (nc + ns) sides per
    stage: the same lengths as the oracle's assembled QP."""
    from paper_2003_02547_gb300.batch import QpBatch
    qps = [soft_qp(0), W.small_random_qp(1), soft_qp(2)]
    b = QpBatch(qps, device=None)
    for i, qp in enumerate(qps):
        dq = O.assemble(qp)
        off = b.offsets(i)
        assert off[4] == dq.ny and off[5] == dq.neq and off[6] == dq.nside and off[7] == dq.nside


def test_slack_data_roundtrip(gqmod):
    from paper_2003_02547_gb300.batch import QpBatch
    qp = soft_qp(3)
    qp.zl[3] = np.array([0.1, 0.2, 0.3, 0.4])
    qp.lus[3] = np.array([0.0, -1.0, 0.5, 2.0])
    b = QpBatch([qp], device=None, share=False)   # stage 3 no longer equals stage 1
    back = b.to_ocp(0)
    for n in range(qp.N + 1):
        assert back.ns(n) == qp.ns(n)
        for f in ("idxs", "Zl", "Zu", "zl", "zu", "lls", "lus"):
            np.testing.assert_array_equal(np.asarray(getattr(back, f)[n]), np.asarray(getattr(qp, f)[n]))


def test_soft_qps_are_scheduled_in_the_block_kernel(gqmod):
    """The one-warp kernel has no slack elimination: a QP with slacks goes to
    the block bucket even when its stages fit a warp."""
    from paper_2003_02547_gb300.batch import QpBatch
    b = QpBatch([W.small_random_qp(0), soft_qp(1), W.small_random_qp(2)], device=None)
    sch = b.schedule()
    assert sch.warp_qps == 2 and sch.block_qps == 1


def test_soft_setter_validates(gqmod):
    gq = gqmod
    from paper_2003_02547_gb300.batch import QpBatch
    b = QpBatch([soft_qp(0)], device=None)
    L = b.lib
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    PI = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    ones = np.ones(4)

    def call(idx, Z=ones, ls=ones):
        return L.gq_set_soft(b.h, 0, 1, PI(np.asarray(idx, dtype=np.int32)), P(Z), P(ones), P(ones), P(ones),
                             P(ls), P(ones))
    assert call([0, 1, 2, 3]) == gq.GQ_OK
    assert call([0, 1, 1, 3]) == gq.GQ_ERR_ARG          # repeated constraint
    assert call([0, 1, 2, 9]) == gq.GQ_ERR_ARG          # out of range (nc = 6 at stage 1)
    assert call([0, 1, 2, 3], Z=np.array([1.0, -1.0, 1.0, 1.0])) == gq.GQ_ERR_DATA
    assert call([0, 1, 2, 3], ls=np.array([1.0, np.inf, 1.0, 1.0])) == gq.GQ_ERR_DATA


def test_stage_ns_is_validated(gqmod):
    gq = gqmod
    from paper_2003_02547_gb300.batch import dims_of
    qp = W.small_random_qp(0)
    dims = dims_of([qp])
    ns = np.zeros(qp.N + 1, dtype=np.int32)
    ns[2] = 7                                             # stage 2 has 6 constraints
    L = gq.load()
    mem = L.gq_batch_memsize(1, dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), dims.size, None)
    buf = np.zeros(mem + 64, dtype=np.uint8)
    ptr = buf.ctypes.data + (-buf.ctypes.data) % 64
    h = ctypes.c_void_p()
    rc = L.gq_batch_create_soft(1, dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), dims.size, None,
                                ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ptr, mem, ctypes.byref(h))
    assert rc == gq.GQ_ERR_DIMS


def test_condensing_rejects_soft_qps(gqmod):
    gq = gqmod
    from paper_2003_02547_gb300.batch import QpBatch
    b = QpBatch([soft_qp(0)], device=None)
    n = ctypes.c_size_t()
    assert b.lib.gq_condense_dims(b.h, 0, 2, None, 0, ctypes.byref(n)) == gq.GQ_ERR_ARG


def test_unset_slack_data_defaults_to_a_consistent_map(gqmod):
    """Before gq_set_soft, slack k relaxes constraint k (zero cost), so the
    kernels never meet an inconsistent slack map."""
    from paper_2003_02547_gb300.batch import QpBatch
    qp = soft_qp(0)
    b = QpBatch([qp], device=None, set_data=False)
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for n in range(qp.N + 1):
        m = qp.ns(n)
        ns = ctypes.c_int()
        idx = np.full(max(m, 1), -7, dtype=np.int32)
        vals = [np.full(max(m, 1), 3.0) for _ in range(6)]
        assert b.lib.gq_get_soft(b.h, 0, n, ctypes.byref(ns), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 *[P(v) for v in vals]) == 0
        assert ns.value == m
        if m:
            np.testing.assert_array_equal(idx[:m], np.arange(m))
            for v in vals:
                assert np.all(v[:m] == 0.0)
