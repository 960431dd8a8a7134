"""gq_solve_noalloc: the solve for callers that cannot allocate device memory.

Such callers (fixed memory budgets, allocators owned by a host application)
pass their own input and solution buffers; the workspace is a static device
array inside the library.  The test compares two consecutive calls of the
no-allocation entry point with gq_solve on the same inputs, through the C ABI.
This file is collected last so that a failure here never hides another test.
"""
import ctypes

import numpy as np
import pytest

from paper_2003_02547_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SOL_TOL = 1e-6   # the solution tolerance of the other GPU parity tests


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2003_02547_gb300 import build
    build.build()
    from paper_2003_02547_gb300 import gq
    from paper_2003_02547_gb300.batch import QpBatch
    return gq, QpBatch, torch


def _rel(a, b):
    return float(np.max(np.abs(a - b), initial=0.0) / max(1.0, np.max(np.abs(b), initial=0.0)))


def _noalloc_solve(env, b, arg):
    """Caller-owned input/solution buffers, static library workspace."""
    gq, QpBatch, torch = env
    dev_in = torch.empty_like(b.dev_in)
    dev_sol = torch.zeros_like(b.dev_sol)
    dev_in.copy_(torch.from_numpy(b.host_in._np[b.host_in.off:b.host_in.off + b.dev_in.numel()]))
    stream = torch.cuda.current_stream()
    rc = b.lib.gq_solve_noalloc(b.h, ctypes.byref(arg), dev_in.data_ptr(), dev_sol.data_ptr(), stream.cuda_stream)
    gq.check(rc)
    torch.cuda.synchronize()
    return dev_sol.cpu().numpy().view(np.float64)


def test_noalloc_matches_solve_on_two_calls(env):
    gq, QpBatch, torch = env
    for prec in (gq.PREC_MIXED, gq.PREC_FP64):
        qps = [W.mass_spring_qp(i) for i in range(12)] + [W.small_random_qp(i) for i in range(4)]
        b = QpBatch(qps)
        assert b.sizes.ws_bytes <= gq.NOALLOC_SCRATCH_BYTES
        arg = gq.default_arg(gq.MODE_SPEED, prec)
        b.upload()
        b.solve(arg)
        b.download()
        torch.cuda.synchronize()
        ref = [b.solution(i) for i in range(len(qps))]
        ref_stats = b.all_stats()
        assert np.all(ref_stats["status"] == 0)
        for call in range(2):
            buf = _noalloc_solve(env, b, arg)
            stats = buf[:b.nqp * 8].view(np.int32).reshape(b.nqp, 16)
            assert np.all(stats[:, 0] == 0), (call, stats[:, 0])
            for i in range(len(qps)):
                got = b.solution(i, buf)
                for g, r in zip(got, ref[i]):
                    assert _rel(g, r) <= SOL_TOL, (prec, call, i)


def test_noalloc_rejects_batches_beyond_the_scratch(env):
    gq, QpBatch, torch = env
    b = QpBatch([W.mass_spring_qp(i) for i in range(400)], set_data=False)
    assert b.sizes.ws_bytes > gq.NOALLOC_SCRATCH_BYTES
    arg = gq.default_arg(gq.MODE_SPEED, gq.PREC_MIXED)
    rc = b.lib.gq_solve_noalloc(b.h, ctypes.byref(arg), b.dev_in.data_ptr(), b.dev_sol.data_ptr(), None)
    assert rc == gq.GQ_ERR_SIZE
    assert "static scratch" in b.lib.gq_last_error().decode()
