"""gq_solve_noalloc: the solve for callers that cannot allocate device memory.

Such callers (fixed memory budgets, allocators owned by a host application,
solves issued where an allocation would synchronise the device) pass their
own input and solution buffers; the workspace is a static device array inside
the library.  Through the C ABI, the test checks that two consecutive calls
of the no-allocation entry point give the same bits as gq_solve on the same
inputs, after the shared array was left full of another batch's data, and
that a call takes no device memory.  This file is collected last so that a
failure here never hides another test.
"""
import ctypes

import numpy as np
import pytest

from paper_2003_02547_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2003_02547_gb300 import build
    build.build()
    from paper_2003_02547_gb300 import gq
    from paper_2003_02547_gb300.batch import QpBatch
    return gq, QpBatch, torch


def _caller_buffers(env, b):
    gq, QpBatch, torch = env
    dev_in = torch.empty_like(b.dev_in)
    dev_sol = torch.zeros_like(b.dev_sol)
    dev_in.copy_(torch.from_numpy(b.host_in._np[b.host_in.off:b.host_in.off + b.dev_in.numel()]))
    torch.cuda.synchronize()
    return dev_in, dev_sol


def _noalloc_call(env, b, arg, dev_in, dev_sol):
    gq, QpBatch, torch = env
    stream = torch.cuda.current_stream()
    rc = b.lib.gq_solve_noalloc(b.h, ctypes.byref(arg), dev_in.data_ptr(), dev_sol.data_ptr(), stream.cuda_stream)
    gq.check(rc)
    torch.cuda.synchronize()
    return dev_sol.cpu().numpy().view(np.float64)


def _fill_scratch_with_other_data(env):
    """Leave the static array full of a different batch's workspace: ragged
    QPs with general constraints solved in FP64 write more of the array than
    the mass-spring batch below uses."""
    gq, QpBatch, torch = env
    qps = [W.ragged_random_qp(i) for i in (17, 44, 46, 47, 53)]
    b = QpBatch(qps)
    assert b.sizes.ws_bytes <= gq.noalloc_scratch_bytes()
    b.upload()
    dev_in, dev_sol = _caller_buffers(env, b)
    buf = _noalloc_call(env, b, gq.default_arg(gq.MODE_SPEED, gq.PREC_FP64), dev_in, dev_sol)
    stats = buf[:b.nqp * 8].view(np.int32).reshape(b.nqp, 16)
    assert np.all(stats[:, 0] == 0), stats[:, 0]
    return b.sizes.ws_bytes


def test_noalloc_matches_solve_bitwise_on_two_calls(env):
    gq, QpBatch, torch = env
    for prec in (gq.PREC_MIXED, gq.PREC_FP64):
        qps = [W.mass_spring_qp(i) for i in range(12)] + [W.small_random_qp(i) for i in range(4)]
        b = QpBatch(qps)
        filled = _fill_scratch_with_other_data(env)
        assert filled > b.sizes.ws_bytes
        arg = gq.default_arg(gq.MODE_SPEED, prec)
        b.upload()
        b.solve(arg)
        b.download()
        torch.cuda.synchronize()
        ref_stats = b.all_stats()
        assert np.all(ref_stats["status"] == 0)
        ref = b.dev_sol.cpu().numpy().view(np.float64).copy()
        dev_in, dev_sol = _caller_buffers(env, b)
        for call in range(2):
            # the same kernels on the same inputs: identical bits, whatever the
            # array held before
            buf = _noalloc_call(env, b, arg, dev_in, dev_sol)
            assert np.array_equal(buf.view(np.uint64), ref.view(np.uint64)), (prec, call)


def test_noalloc_call_takes_no_device_memory(env):
    gq, QpBatch, torch = env
    b = QpBatch([W.mass_spring_qp(i) for i in range(8)])
    b.upload()
    arg = gq.default_arg(gq.MODE_SPEED, gq.PREC_MIXED)
    dev_in, dev_sol = _caller_buffers(env, b)
    _noalloc_call(env, b, arg, dev_in, dev_sol)   # warm-up: first call per device looks up the array
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _noalloc_call(env, b, arg, dev_in, dev_sol)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0, (free0, free1)


def test_noalloc_rejects_batches_beyond_the_scratch(env):
    gq, QpBatch, torch = env
    b = QpBatch([W.mass_spring_qp(i) for i in range(400)], set_data=False)
    assert b.sizes.ws_bytes > gq.noalloc_scratch_bytes()
    arg = gq.default_arg(gq.MODE_SPEED, gq.PREC_MIXED)
    rc = b.lib.gq_solve_noalloc(b.h, ctypes.byref(arg), b.dev_in.data_ptr(), b.dev_sol.data_ptr(), None)
    assert rc == gq.GQ_ERR_SIZE
    assert "static scratch" in b.lib.gq_last_error().decode()
