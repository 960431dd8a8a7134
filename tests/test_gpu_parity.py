"""CUDA path against the CPU oracle, through the C ABI (GPU required).

Tolerances (stated here, used below):
* FP64 row-level checks (residuals, one Newton direction): relative 1e-9 of
  the largest entry -- both sides solve the same linear system in FP64, the
  difference is rounding order times the condition number of eq. (kkt) at a
  moderate iterate.
* converged solutions: KKT residual norms recomputed on the CPU <= 1e-8 (the
  exit rule), and ||y - y*||inf / max(1, ||y*||inf) <= 1e-6 against the
  oracle run with the SAME exit rule from the same start (same algorithm in
  FP64, same trajectory).  Against the oracle run to 1e-10 the distance is
  only bounded by 2e-3: at a degenerate bound (lambda* = 0 and t* = 0)
  mu = 1e-8 allows t ~ sqrt(mu) = 1e-4, and the mass-spring batch has such
  bounds (observed distances up to 1.04e-3).
* iterates after k IPM iterations (FP64): relative 1e-8.
* mixed path: same gates as FP64 after refinement.
"""
import numpy as np
import pytest

import test_oracle_pins as P
from oracle import ocp_ipm as O
from paper_2003_02547_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SOL_TOL = 1e-6
EXACT_TOL = 2e-3
KKT_TOL = 1e-8
SAME_RULE = dict(tol_stat=1e-8, tol_eq=1e-8, tol_ineq=1e-8, tol_comp=1e-8)


def oracle_pair(qp, warm=None):
    """(same-exit-rule oracle from the same start, tightly converged oracle);
    warm = (y, pi, lam, t) for a primal-dual warm start."""
    if warm is not None:
        same = O.solve(qp, O.IpmArg(warm_start=2, **SAME_RULE), *warm)
    else:
        same = O.solve(qp, O.IpmArg(**SAME_RULE))
    return same, O.solve(qp)


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2003_02547_gb300 import build
    build.build()
    from paper_2003_02547_gb300 import gq
    from paper_2003_02547_gb300.batch import QpBatch
    return gq, QpBatch, torch


def solve_gpu(env, qps, precision=0, mode=0, share=True, **argover):
    gq, QpBatch, torch = env
    b = QpBatch(qps, share=share)
    arg = gq.default_arg(mode, precision, **argover)
    b.upload()
    b.solve(arg)
    b.download()
    torch.cuda.synchronize()
    return b


def rel_err(a, b):
    return float(np.max(np.abs(a - b), initial=0.0) / max(1.0, np.max(np.abs(b), initial=0.0)))


def mixed_set():
    """Stage-varying sizes, S != 0, nx_0 > 0, general rows, masked sides."""
    out = []
    for seed in range(4):
        qp = P.random_lq(300 + seed, N=6, boxes=True, ng=2, tight=0.8)
        qp.lbu[2] = np.full(len(qp.lbu[2]), -np.inf)
        qp.ug[3] = np.full(len(qp.ug[3]), np.inf)
        qp.validate()
        out.append(qp)
    return out


def random_iterate(qp, dq, seed):
    rng = np.random.default_rng(seed)
    y = rng.standard_normal(dq.ny)
    pi = rng.standard_normal(dq.neq)
    lam = rng.uniform(0.2, 2.0, dq.nside)
    t = rng.uniform(0.2, 2.0, dq.nside)
    lam[~dq.active] = 0.0
    t[~dq.active] = 1.0
    return y, pi, lam, t


# ----------------------------------------------------------------------------
# a1: residuals
# ----------------------------------------------------------------------------
def test_residual_norms_match_oracle(env):
    gq, QpBatch, torch = env
    qps = mixed_set() + [W.small_random_qp(0), W.mass_spring_qp(0)]
    b = QpBatch(qps)
    its = []
    for i, qp in enumerate(qps):
        dq = O.assemble(qp)
        it = random_iterate(qp, dq, i)
        its.append((dq, it))
        b.set_guess(i, *it)
    b.upload()
    b.upload_sol()
    b.residuals()
    b.download()
    torch.cuda.synchronize()
    st = b.all_stats()
    for i, (dq, (y, pi, lam, t)) in enumerate(its):
        rg, rb, rd, mu = O.residuals(dq, y, pi, lam[dq.active], t[dq.active])
        ref = [np.max(np.abs(rg)), np.max(np.abs(rb), initial=0), np.max(np.abs(rd)), mu]
        np.testing.assert_allclose(st["res"][i], ref, rtol=1e-12, atol=1e-14)


# ----------------------------------------------------------------------------
# a2-a4: one Newton direction through the Riccati factorisation
# ----------------------------------------------------------------------------
def _newton_compare(env, qps, precision, ir_steps, tol, sigma_mu=0.37, ir_tol=None, mode=0, schedule=None):
    gq, QpBatch, torch = env
    b = QpBatch(qps)
    if schedule is not None:
        b.set_schedule(*schedule)
    its = []
    for i, qp in enumerate(qps):
        dq = O.assemble(qp)
        it = random_iterate(qp, dq, 100 + i)
        its.append((dq, it))
        b.set_guess(i, *it)
    b.upload()
    b.upload_sol()
    out = torch.zeros_like(b.dev_sol)
    arg = gq.default_arg(mode, precision, ir_steps=ir_steps)
    if ir_tol is not None:
        arg.ir_tol = ir_tol
    b.newton_step(arg, sigma_mu, out)
    torch.cuda.synchronize()
    buf = out.cpu().numpy().view(np.float64)
    worst = 0.0
    for i, (dq, (y, pi, lam, t)) in enumerate(its):
        a = dq.active
        dy, dpi, dlam, dt = O.newton_step(dq, y, pi, lam[a], t[a], sigma_mu=sigma_mu)
        gy, gpi, glam, gt = b.solution(i, buf)
        for g, r in ((gy, dy), (gpi, dpi), (glam[a], dlam), (gt[a], dt)):
            worst = max(worst, float(np.max(np.abs(g - r), initial=0) / max(1e-300, np.max(np.abs(r), initial=1))))
        assert np.all(glam[~a] == 0.0) and np.all(gt[~a] == 0.0)
    assert worst <= tol, worst
    return worst


def test_newton_step_fp64_matches_oracle(env):
    qps = mixed_set() + [W.small_random_qp(1), W.mass_spring_qp(1), W.ragged_random_qp(5)]
    _newton_compare(env, qps, precision=0, ir_steps=0, tol=1e-9)


def test_newton_step_mixed_without_refinement_is_fp32_accurate(env):
    qps = [W.small_random_qp(1), W.mass_spring_qp(1)]
    w = _newton_compare(env, qps, precision=1, ir_steps=0, tol=1e-3)
    assert w > 1e-12   # it really ran in FP32


def test_newton_step_mixed_with_refinement_matches_oracle(env):
    qps = [W.small_random_qp(1), W.mass_spring_qp(1)] + mixed_set()[:2]
    _newton_compare(env, qps, precision=1, ir_steps=4, tol=1e-9, ir_tol=1e-12)


def test_newton_step_tensor_core_products_match_oracle(env):
    """Large stages (nu + nx = 192, nx = 128): the FP32 factor's products run
    on the tcgen05 tensor cores (3xTF32, accumulators in TMEM).  One Newton
    direction with refinement equals the oracle's at random iterates, and
    without refinement it is within the FP32 factor's accuracy."""
    qps = [W.large_stage_qp(i, N=3) for i in range(2)]
    _newton_compare(env, qps, precision=1, ir_steps=6, tol=1e-9, ir_tol=1e-13)
    _newton_compare(env, qps, precision=1, ir_steps=0, tol=1e-3)


# ----------------------------------------------------------------------------
# full IPM
# ----------------------------------------------------------------------------
def _check_converged(b, qps, refs, sol_tol=SOL_TOL):
    """refs[i] is None or a pair from oracle_pair()."""
    st = b.all_stats()
    for i, qp in enumerate(qps):
        assert st["status"][i] == 0, (i, st[i])
        y, pi, lam, t = b.solution(i)
        kkt = O.full_residuals(qp, y, pi, lam, t)
        assert max(kkt[:4]) <= KKT_TOL * 1.01, (i, kkt)
        assert np.all(lam >= 0) and np.all(t > 0)
        if refs is not None and refs[i] is not None:
            same, tight = refs[i]
            assert same.status == O.CONVERGED
            assert rel_err(y, same.y) <= sol_tol, (i, rel_err(y, same.y), st["iters"][i], same.iters)
            # the 1e-10 oracle itself may stop on a tiny step in the end game
            if tight.status == O.CONVERGED:
                assert rel_err(y, tight.y) <= EXACT_TOL, (i, rel_err(y, tight.y))


def test_ipm_fp64_matches_oracle_small(env):
    qps = [W.small_random_qp(i) for i in range(4)] + mixed_set()
    refs = [oracle_pair(q) for q in qps]
    b = solve_gpu(env, qps, precision=0)
    _check_converged(b, qps, refs)


def test_ipm_fp64_matches_oracle_ragged(env):
    qps = [W.ragged_random_qp(i) for i in range(3)]
    refs = [oracle_pair(q) for q in qps]
    b = solve_gpu(env, qps, precision=0)
    _check_converged(b, qps, refs)


def test_ipm_iterates_match_oracle(env):
    """Same algorithm step by step: iterates after k iterations agree."""
    qps = [W.small_random_qp(2), W.mass_spring_qp(2)] + mixed_set()[:2]
    for k in (1, 2, 3):
        b = solve_gpu(env, qps, precision=0, iter_max=k, tol_stat=0.0, tol_eq=0.0, tol_ineq=0.0, tol_comp=0.0)
        for i, qp in enumerate(qps):
            ref = O.solve(qp, O.IpmArg(iter_max=k, tol_stat=0, tol_eq=0, tol_ineq=0, tol_comp=0))
            y, pi, lam, t = b.solution(i)
            assert b.all_stats()["iters"][i] == k
            assert rel_err(y, ref.y) <= 1e-8, (k, i)
            assert rel_err(pi, ref.pi) <= 1e-8, (k, i)
            assert rel_err(lam, ref.lam) <= 1e-8, (k, i)
            assert rel_err(t, ref.t) <= 1e-8, (k, i)


def test_ipm_mixed_matches_oracle(env):
    qps = [W.small_random_qp(0)] + [W.mass_spring_qp(i) for i in range(6)] + mixed_set()[:2]
    refs = [oracle_pair(q) for q in qps]
    b = solve_gpu(env, qps, precision=1)
    _check_converged(b, qps, refs)


def test_unconstrained_is_one_newton_step(env):
    qps = [P.random_lq(s, N=6) for s in range(3)]
    b = solve_gpu(env, qps, precision=0)
    st = b.all_stats()
    for i, qp in enumerate(qps):
        assert st["status"][i] == 0 and st["iters"][i] == 1
        us, xs, pis = P.riccati_dp(qp)
        y, pi, _, _ = b.solution(i)
        ref = np.concatenate([np.concatenate([us[n], xs[n]]) for n in range(qp.N + 1)])
        np.testing.assert_allclose(y, ref, rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(pi, np.concatenate(pis), rtol=1e-9, atol=1e-10)


def test_batch_invariance_bitwise(env):
    """A QP gives the same bits alone and inside a ragged batch."""
    target = W.mass_spring_qp(7)
    mix = [W.ragged_random_qp(i) for i in range(4)] + [target] + [W.small_random_qp(3)]
    for prec in (0, 1):
        alone = solve_gpu(env, [target], precision=prec)
        inmix = solve_gpu(env, mix, precision=prec)
        for a, b_ in zip(alone.solution(0), inmix.solution(4)):
            np.testing.assert_array_equal(a, b_)
        assert alone.all_stats()["iters"][0] == inmix.all_stats()["iters"][4]


def test_stale_workspace_and_solution_buffers_do_not_matter(env):
    """A cold solve reads nothing it did not write: the same bits with zeroed
    and with NaN-filled workspace and solution buffers (the server reuses
    its lanes' buffers without clearing them)."""
    gq, QpBatch, torch = env
    qps = [W.ragged_random_qp(i) for i in range(3)] + [W.mass_spring_qp(2), W.small_random_qp(5)]
    for prec in (0, 1):
        arg = gq.default_arg(0, prec)
        ref = solve_gpu(env, qps, precision=prec)
        b = QpBatch(qps)
        b.dev_ws.fill_(0xFF)
        b.dev_sol.fill_(0xFF)
        b.upload()
        b.solve(arg)
        b.download()
        torch.cuda.synchronize()
        for i in range(len(qps)):
            for a, c in zip(ref.solution(i), b.solution(i)):
                np.testing.assert_array_equal(a, c, err_msg=f"precision {prec}, QP {i}")
            assert ref.all_stats()["iters"][i] == b.all_stats()["iters"][i]


def test_status_paths_do_not_poison_neighbours(env):
    gq, QpBatch, torch = env
    good = W.small_random_qp(0)
    rng = np.random.default_rng([7, 7])
    bad = P.random_lq(107, N=2, nxs=[0, 2, 2], nus=[1, 1, 0], boxes=True, tight=0.35)
    bad.idxbx[2] = bad.idxbx[2][:1]
    bad.lbx[2] = bad.lbx[2][:1]
    bad.ubx[2] = bad.ubx[2][:1]
    bad.C[1] = rng.standard_normal((1, 2))
    bad.D[1] = rng.standard_normal((1, 1))
    bad.lg[1] = np.array([-0.3])
    bad.ug[1] = np.array([0.4])
    assert P.brute_force(bad) is None          # infeasible
    b = solve_gpu(env, [good, bad, good], precision=0, iter_max=60)
    st = b.all_stats()
    assert st["status"][0] == 0 and st["status"][2] == 0
    assert st["status"][1] in (1, 2, 3)
    np.testing.assert_array_equal(b.solution(0)[0], b.solution(2)[0])
    # iteration cap and device timeout end every QP with its own status
    b = solve_gpu(env, [good], precision=0, iter_max=0)
    assert b.all_stats()["status"][0] == 1
    b = solve_gpu(env, [good, W.mass_spring_qp(0)], precision=0, timeout_ns=1)
    assert list(b.all_stats()["status"]) == [4, 4]


def test_warm_start_converges_faster(env):
    gq, QpBatch, torch = env
    qp = W.ragged_random_qp(11)
    cold = solve_gpu(env, [qp], precision=0)
    y, pi, lam, t = cold.solution(0)
    qp2 = W.perturb_x0(qp, qp.x0 + 0.01 * np.random.default_rng(0).standard_normal(qp.x0.shape))
    b = QpBatch([qp2])
    b.set_guess(0, y, pi, lam, t)
    b.upload()
    b.upload_sol()
    b.solve(gq.default_arg(0, 0, warm_start=2))
    b.download()
    torch.cuda.synchronize()
    _check_converged(b, [qp2], [oracle_pair(qp2, warm=(y, pi, lam, t))])
    assert b.all_stats()["iters"][0] < cold.all_stats()["iters"][0]


@pytest.mark.parametrize("precision", [1, 0])
def test_mass_spring_full_batch(env, precision):
    """The timed workload: 1024 mass-spring QPs, one launch.  Every QP is
    checked through KKT residuals recomputed on the CPU; a sample against
    the oracle's solution."""
    qps = W.mass_spring_batch(1024)
    b = solve_gpu(env, qps, precision=precision)
    sample = set(range(0, 1024, 97)) | {1023}
    refs = [oracle_pair(q) if i in sample else None for i, q in enumerate(qps)]
    _check_converged(b, qps, refs)
    if precision == 1:
        # the FP32 factors plus refinement suffice on this workload: a QP
        # handed to FP64 would mean inaccurate FP32 factors
        assert not np.any(b.all_stats()["flags"] & 1)


def test_schedules_agree_and_autotune_picks_one(env):
    """The same QPs solved one per warp and one per block (two different
    kernels) meet the same oracle gates; the autotuner returns one of its
    candidate schedules and leaves the batch solving correctly."""
    gq, QpBatch, torch = env
    qps = [W.mass_spring_qp(i) for i in range(3)] + [W.small_random_qp(1)]
    refs = [oracle_pair(q) for q in qps]
    for prec in (1, 0):
        arg = gq.default_arg(0, prec)
        sols = []
        for wmax, thr in ((32, 256), (0, 256), (0, 128)):
            b = QpBatch(qps)
            b.set_schedule(wmax, thr)
            b.upload()
            b.solve(arg)
            b.download()
            torch.cuda.synchronize()
            sch = b.schedule()
            assert sch.warp_qps == (len(qps) if wmax else 0)
            _check_converged(b, qps, refs)
            sols.append([b.solution(i)[0] for i in range(len(qps))])
        for other in sols[1:]:
            for y0, y1 in zip(sols[0], other):
                assert rel_err(y1, y0) <= 1e-6
        b = QpBatch(qps)
        b.upload()
        sch, ms = b.autotune(arg, reps=2)
        assert sch.warp_max_nv in (32, 24, 16, 0) and sch.block_threads in (256, 128, 64) and ms > 0
        assert sch.tensor_cores in (0, 2)
        b.solve(arg)
        b.download()
        torch.cuda.synchronize()
        _check_converged(b, qps, refs)


def test_solve_replays_from_a_cuda_graph(env):
    """A solve call (mirror copy, FP32 launch, FP64 continuation launch) is
    captured in a CUDA graph; each replay gives the bits of a direct solve."""
    gq, QpBatch, torch = env
    qps = [W.small_random_qp(0), W.mass_spring_qp(3)]
    arg = gq.default_arg(0, 1)
    ref = solve_gpu(env, qps, precision=1)
    b = QpBatch(qps)
    b.upload()
    b.solve(arg)          # first call outside the capture (launch attributes)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.solve(arg)
    for _ in range(3):
        b.dev_sol.zero_()
        g.replay()
    b.download()
    torch.cuda.synchronize()
    for i in range(len(qps)):
        for a, c in zip(ref.solution(i), b.solution(i)):
            np.testing.assert_array_equal(a, c)


def _solve_sched(env, qps, precision, riccati, wmax=0):
    gq, QpBatch, torch = env
    b = QpBatch(qps)
    b.set_schedule(wmax, 256)
    b.upload()
    b.solve(gq.default_arg(0, precision, riccati=riccati))
    b.download()
    torch.cuda.synchronize()
    return b


def test_classical_riccati_solves_indefinite_state_cost(env):
    """NEXT-1: with an indefinite Q (reduced Hessians positive definite) the
    square-root factorisation has no Cholesky factor and the QP ends NaN;
    the classical variant converges to the oracle's solution."""
    gq, QpBatch, torch = env
    qps = [P.indefinite_lq(s) for s in range(3)]
    refs = [oracle_pair(q) for q in qps]
    for prec in (0, 1):
        sq = _solve_sched(env, qps, prec, 0)
        assert np.all(sq.all_stats()["status"] == gq.STATUS_NAN)
        cl = _solve_sched(env, qps, prec, 1)
        _check_converged(cl, qps, refs)


def test_classical_riccati_matches_square_root_on_convex_qps(env):
    """On strictly convex QPs both variants reach the oracle's solution."""
    gq, QpBatch, torch = env
    qps = [W.small_random_qp(2), W.mass_spring_qp(4)] + mixed_set()[:2] + [W.ragged_random_qp(1)]
    refs = [oracle_pair(q) for q in qps]
    for prec in (0, 1):
        cl = _solve_sched(env, qps, prec, 1)
        _check_converged(cl, qps, refs)
    b = QpBatch(qps)          # default schedule: warp bucket present
    with pytest.raises(gq.GqError) as e:
        b.solve(gq.default_arg(0, 0, riccati=1))
    assert e.value.code == gq.GQ_ERR_ARG


@pytest.mark.parametrize("warp_max_nv", [32, 0])
def test_robust_mode_array_algorithm_matches_oracle(env, warp_max_nv):
    """Mode robust (Sec. 4.2): every Riccati factor from the QR array
    algorithm, in the one-warp kernel (QPs with nv <= 32) and in the block
    kernel (warp_max_nv = 0: all QPs).  One Newton direction at random
    iterates equals the oracle's (FP64, 1e-9), and full solves meet the
    oracle gates in both precisions."""
    gq, QpBatch, torch = env
    qps = [W.small_random_qp(2), W.mass_spring_qp(4)] + mixed_set()[:2] + [W.ragged_random_qp(1)]
    _newton_compare(env, qps, precision=0, ir_steps=0, tol=1e-9, mode=2, schedule=(warp_max_nv, 256))
    refs = [oracle_pair(q) for q in qps]
    for prec in (0, 1):
        b = QpBatch(qps)
        b.set_schedule(warp_max_nv, 256)
        b.upload()
        b.solve(gq.default_arg(2, prec))
        b.download()
        torch.cuda.synchronize()
        _check_converged(b, qps, refs)


@pytest.mark.parametrize("warp_max_nv", [32, 0])
def test_balance_mode_switches_to_array_algorithm(env, warp_max_nv):
    """Mode balance (Sec. 4.2): a direction that refinement cannot make
    accurate repeats the factorisation with the array algorithm.  With
    ir_fail_ratio = 0 every refined direction counts as inaccurate, so every
    QP takes the whole chain (mixed: FP32 -> FP64 factors -> array
    algorithm; FP64: Cholesky -> array algorithm) and must still meet the
    oracle gates."""
    gq, QpBatch, torch = env
    qps = [W.small_random_qp(i) for i in range(2)] + [W.mass_spring_qp(3)] + mixed_set()[:2] \
        + [W.ragged_random_qp(1)]
    refs = [oracle_pair(q) for q in qps]
    for prec in (0, 1):
        b = QpBatch(qps)
        b.set_schedule(warp_max_nv, 256)
        b.upload()
        b.solve(gq.default_arg(1, prec, ir_fail_ratio=0.0))
        b.download()
        torch.cuda.synchronize()
        fl = b.all_stats()["flags"]
        assert np.all(fl & gq.FLAG_ARRAY_QR), fl
        if prec == 1:
            assert np.all(fl & gq.FLAG_FP64_FALLBACK), fl
        _check_converged(b, qps, refs)
