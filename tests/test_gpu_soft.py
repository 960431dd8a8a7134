"""Soft constraints (Sec. 2.2) on the GPU against the oracle.

The CUDA path eliminates the slacks inside the block kernel (per-slack
diagonal elimination folded into the barrier terms); the oracle keeps them
as ordinary primal variables with their own sides.  Gates as in
test_gpu_parity: one Newton direction at random iterates to 1e-9 (FP64),
full solves converged with CPU-recomputed KKT residuals <= 1e-8 and y
(slacks included) within 1e-6 of the same-exit-rule oracle (strictly convex
slack costs, Z > 0, so the solution is unique).
"""
import numpy as np
import pytest

import test_gpu_parity as GP
from test_gpu_parity import env  # noqa: F401  (shared module fixture)
from oracle import ocp_ipm as O
from paper_2003_02547_gb300 import workloads as W

pytestmark = pytest.mark.gpu

_REFS = {}


def refs_for(qps):
    """Oracle references (same exit rule, tight), computed once per QP."""
    out = []
    for q in qps:
        if q.name not in _REFS:
            _REFS[q.name] = GP.oracle_pair(q)
        out.append(_REFS[q.name])
    return out


def soft_set():
    """Soft state boxes, soft input boxes, soft general rows (with masked
    sides), negative slack bounds, and a ragged QP with every constraint
    soft."""
    a = W.soften(W.small_random_qp(1, x0_scale=2.0), range(1, 11), "x", Z=2.0, z=0.3, ls=0.0)
    b = W.soften(W.small_random_qp(2, x0_scale=2.0), range(0, 10), "u", Z=0.5, z=1.0, ls=-0.05)
    g = W.soften(GP.mixed_set()[0], range(0, 7), "g", Z=1.0, z=0.2, ls=0.0)
    r = W.soften(W.ragged_random_qp(3), range(0, W.ragged_random_qp(3).N + 1), "all", Z=3.0, z=0.1, ls=0.0)
    return [a, b, g, r]


def test_soft_newton_step_fp64_matches_oracle(env):
    GP._newton_compare(env, soft_set(), precision=0, ir_steps=0, tol=1e-9)


def test_soft_newton_step_mixed_with_refinement_matches_oracle(env):
    GP._newton_compare(env, soft_set()[:3], precision=1, ir_steps=4, tol=1e-9, ir_tol=1e-12)


@pytest.mark.parametrize("precision", [0, 1])
def test_soft_solve_matches_oracle(env, precision):
    qps = soft_set()
    refs = refs_for(qps)
    b = GP.solve_gpu(env, qps, precision=precision)
    GP._check_converged(b, qps, refs)
    # the slacks are open somewhere (the soft problem differs from the hard one)
    opened = 0
    for i, qp in enumerate(qps):
        dq = O.assemble(qp)
        y = b.solution(i)[0]
        opened += sum(int(np.max(np.concatenate(p) - np.concatenate([qp.lls[n], qp.lus[n]]), initial=0) > 1e-4)
                      for n, p in enumerate(O.split_slacks(qp, dq, y)))
    assert opened > 0


def test_soft_and_hard_qps_in_one_batch(env):
    """Hard QPs run in the one-warp kernel and soft QPs in the block kernel
    of the same solve call; both meet the oracle gates."""
    gq, QpBatch, torch = env
    qps = [W.small_random_qp(4), soft_set()[0], W.mass_spring_qp(2), soft_set()[2]]
    b = QpBatch(qps)
    sch = b.schedule()
    assert sch.warp_qps == 2 and sch.block_qps == 2
    refs = refs_for(qps)
    for prec in (0, 1):
        b.upload()
        b.solve(gq.default_arg(0, prec))
        b.download()
        torch.cuda.synchronize()
        GP._check_converged(b, qps, refs)


def test_exact_l1_penalty_on_gpu(env):
    """Exact penalty: Z = 0 and z above the hard multipliers reproduce the
    hard solution (solved by the GPU too) with zero slacks."""
    hard_qp = W.small_random_qp(3, x0_scale=2.0)
    hb = GP.solve_gpu(env, [hard_qp], precision=0)
    assert hb.all_stats()["status"][0] == 0
    lam = hb.solution(0)[2]
    soft = W.soften(hard_qp, range(hard_qp.N + 1), "all", Z=0.0, z=10.0 * float(np.max(lam)) + 1.0)
    for prec in (0, 1):
        sb = GP.solve_gpu(env, [soft], precision=prec)
        assert sb.all_stats()["status"][0] == 0
        dq_h, dq_s = O.assemble(hard_qp), O.assemble(soft)
        yh, ys = hb.solution(0)[0], sb.solution(0)[0]
        for (uh, xh), (us, xs) in zip(O.split_stages(hard_qp, dq_h, yh), O.split_stages(soft, dq_s, ys)):
            np.testing.assert_allclose(us, uh, atol=1e-6)
            np.testing.assert_allclose(xs, xh, atol=1e-6)
        for sl, su in O.split_slacks(soft, dq_s, ys):
            assert np.all(np.abs(sl) <= 1e-6) and np.all(np.abs(su) <= 1e-6)


def test_soft_relaxes_an_infeasible_problem(env):
    """Hard bounds no input can meet make the hard solve fail; relaxed, the
    GPU converges to the oracle's soft solution."""
    qp = W.small_random_qp(5, x0_scale=2.0)
    qp.lbx[1] = np.full_like(qp.lbx[1], -0.01)
    qp.ubx[1] = np.full_like(qp.ubx[1], 0.01)
    qp.lbu[0] = np.full_like(qp.lbu[0], -0.01)
    qp.ubu[0] = np.full_like(qp.ubu[0], 0.01)
    qp.validate()
    hb = GP.solve_gpu(env, [qp], precision=0)
    assert hb.all_stats()["status"][0] != 0
    soft = W.soften(qp, [1], "x", Z=1.0, z=0.1)
    refs = refs_for([soft])
    for prec in (0, 1):
        GP._check_converged(GP.solve_gpu(env, [soft], precision=prec), [soft], refs)


def test_soft_warm_start_primal_dual(env):
    """A perturbed soft QP warm-started (primal + dual, Sec. 4.2) from the
    previous solution converges to the oracle's solution."""
    gq, QpBatch, torch = env
    qp = soft_set()[0]
    b = GP.solve_gpu(env, [qp], precision=0)
    y, pi, lam, t = b.solution(0)
    qp2 = W.perturb_x0(qp, qp.x0 + 0.01)
    b2 = QpBatch([qp2])
    b2.set_guess(0, y, pi, lam, t)
    b2.upload()
    b2.upload_sol()
    b2.solve(gq.default_arg(0, 0, warm_start=2))
    b2.download()
    torch.cuda.synchronize()
    GP._check_converged(b2, [qp2], [GP.oracle_pair(qp2, warm=(y, pi, lam, t))])
