"""Parity on the ragged and large-stage workloads (GPU required).

Gates (stated here, used below):
* every QP converges (status CONVERGED) within the kernel's exit rule, and
  its KKT residual norms recomputed on the CPU from the returned iterate are
  <= 1e-8 (the unscaled exit rule of the IPM, Sec. 4.2);
* FP64 path: y within 1e-6 (relative to max(1, ||y*||inf)) of the oracle run
  with the same exit rule from the same start -- same algorithm, same
  trajectory;
* mixed path: the trajectory differs from the FP64 one by rounding, and on
  these QPs (general constraints, many weakly active bounds) two points that
  both meet the exit rule can be 1e-3 apart in y (t ~ sqrt(mu) at a
  degenerate bound).  What is unique and well conditioned is the optimal
  value: the primal objective must agree with the oracle's to 1e-6
  relative, and the solution must meet the KKT gate above.
Full-size batches run in the launch configuration of the workload (one
launch over all QPs); the oracle checks a fixed sample of them.
"""
import numpy as np
import pytest

import test_gpu_parity as GP
from test_gpu_parity import env  # noqa: F401  (shared module fixture)
from oracle import ocp_ipm as O
from paper_2003_02547_gb300 import workloads as W

pytestmark = pytest.mark.gpu

OBJ_TOL = 1e-6


def objective_rel(qp, y, ref_y):
    dq = O.assemble(qp)
    f, fs = O.objective(dq, y), O.objective(dq, ref_y)
    return abs(f - fs) / max(1.0, abs(fs))


def check_sample(b, qps, idx, precision):
    st = b.all_stats()
    for i in idx:
        qp = qps[i]
        y, pi, lam, t = b.solution(i)
        kkt = O.full_residuals(qp, y, pi, lam, t)
        assert max(kkt[:4]) <= GP.KKT_TOL * 1.01, (i, kkt)
        same = O.solve(qp, O.IpmArg(**GP.SAME_RULE))
        assert same.status == O.CONVERGED, i
        if precision == 0:
            assert GP.rel_err(y, same.y) <= GP.SOL_TOL, (i, GP.rel_err(y, same.y), st["iters"][i], same.iters)
        assert objective_rel(qp, y, same.y) <= OBJ_TOL, (i, objective_rel(qp, y, same.y))


def test_ragged_mixed_matches_oracle(env):
    qps = [W.ragged_random_qp(i) for i in range(6)]
    b = GP.solve_gpu(env, qps, precision=1)
    st = b.all_stats()
    assert np.all(st["status"] == 0), st
    check_sample(b, qps, range(len(qps)), 1)


@pytest.mark.parametrize("precision", [1, 0])
def test_ragged_full_batch(env, precision):
    """4096 ragged QPs (N ~ U{10..100}, nx ~ U{4..64}, general rows) in one
    solve call, every QP converged, a sample checked against the oracle."""
    qps = W.ragged_batch(4096)
    b = GP.solve_gpu(env, qps, precision=precision)
    st = b.all_stats()
    bad = np.nonzero(st["status"] != 0)[0]
    assert bad.size == 0, (bad[:10], st[bad[:5]])
    check_sample(b, qps, [0, 1, 1000, 2047, 4095], precision)


def test_large_stage_reduced_horizon(env):
    """nx = 128, nu = 64 stages (the large-stage workload) at N = 6, where
    the dense oracle is fast: both precisions against it."""
    qps = [W.large_stage_qp(i, N=6) for i in range(3)]
    for prec in (0, 1):
        b = GP.solve_gpu(env, qps, precision=prec)
        assert np.all(b.all_stats()["status"] == 0), b.all_stats()
        check_sample(b, qps, range(len(qps)), prec)


@pytest.mark.parametrize("precision", [1, 0])
def test_large_stage_full_batch(env, precision):
    """256 QPs with N = 100, nx = 128, nu = 64 in one solve call: every QP
    converged, and the KKT residuals of a sample recomputed on the CPU meet
    the exit rule (two of these QPs are compared with the oracle's sparse
    solve at the full horizon in test_gpu_optimum.py)."""
    qps = W.large_stage_batch(256)
    b = GP.solve_gpu(env, qps, precision=precision)
    st = b.all_stats()
    bad = np.nonzero(st["status"] != 0)[0]
    assert bad.size == 0, (bad[:10], st[bad[:5]])
    for i in (0, 127, 255):
        y, pi, lam, t = b.solution(i)
        kkt = O.full_residuals(qps[i], y, pi, lam, t)
        assert max(kkt[:4]) <= GP.KKT_TOL * 1.01, (i, kkt)
        assert np.all(lam >= 0) and np.all(t > 0)


def test_large_stage_with_and_without_tensor_cores(env):
    """The same large-stage QPs (nu + nx = 192) in the mixed path with the
    tcgen05 products (schedule tensor_cores = 2, and 1 = automatic, which
    takes them for two QPs on a GPU of at least four SMs) and with the
    warp-level mma.sync products (0):
    all meet the oracle gates."""
    gq, QpBatch, torch = env
    qps = [W.large_stage_qp(i, N=6) for i in range(2)]
    for tc in (2, 1, 0):
        b = QpBatch(qps)
        b.set_schedule(32, 256, tc)
        assert b.schedule().tensor_cores == tc
        b.upload()
        b.solve(gq.default_arg(0, 1))
        b.download()
        torch.cuda.synchronize()
        assert np.all(b.all_stats()["status"] == 0), (tc, b.all_stats())
        check_sample(b, qps, range(len(qps)), 1)
