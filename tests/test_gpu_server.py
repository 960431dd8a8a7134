"""Continuous-batching server through the C ABI (GPU required).

The serving contract: every request's result is the same alone and in the
mix.  Cold requests are compared bit for bit with a one-QP batch solved by
gq_solve; a warm repeat is compared bit for bit with a one-QP batch
warm-started (primal + dual, Sec. 4.2) from the previous solution of its key
computed alone.  Bitwise equality holds because every QP's IPM runs in its own
thread block or warp with fixed-order reductions, so neighbours in a
micro-batch cannot change its arithmetic.  Cold results are also checked
against the CPU oracle with the gates of the parity tests.
"""
import numpy as np
import pytest

import test_gpu_parity as GP
from oracle import ocp_ipm as O
from paper_2003_02547_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SOL_TOL = 1e-6
EXACT_TOL = 2e-3


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2003_02547_gb300 import build
    build.build()
    from paper_2003_02547_gb300 import gq, server
    from paper_2003_02547_gb300.batch import QpBatch
    return gq, server, QpBatch, torch


def request_stream(nkeys=10, nrep=2, seed=0):
    """Keys 0..nkeys-1: a cold base QP each (ragged sizes plus two mass-spring
    QPs for the one-warp-per-QP kernel), then `nrep` rounds of warm repeats
    with x0 perturbed by N(0, 0.01^2) (the serving workload's rule)."""
    rng = np.random.default_rng([3, 99, seed])
    base = [W.ragged_random_qp(i) for i in range(nkeys - 2)] + [W.mass_spring_qp(0), W.mass_spring_qp(1)]
    reqs = [(k, base[k], False) for k in range(nkeys)]
    for _ in range(nrep):
        for k in range(nkeys):
            x0 = base[k].x0 + 0.01 * rng.standard_normal(base[k].x0.shape)
            reqs.append((k, W.perturb_x0(base[k], x0), True))
    return reqs


def solve_alone(env, qp, arg, warm=None):
    gq, _, QpBatch, torch = env
    b = QpBatch([qp])
    b.upload()
    a = gq.IpmArg.from_buffer_copy(arg)
    if warm is not None:
        b.set_guess(0, *warm)
        b.upload_sol()
        a.warm_start = 2
    b.solve(a)
    b.download()
    torch.cuda.synchronize()
    return b.solution(0), b.stats(0)


@pytest.mark.parametrize("precision", [1, 0])
def test_same_alone_and_in_the_mix(env, precision):
    gq, server, QpBatch, torch = env
    reqs = request_stream()
    arg = gq.default_arg(0, precision)
    # alone: each request in its own one-QP batch, warm chains per key
    alone, last = [], {}
    for k, qp, warm in reqs:
        sol, st = solve_alone(env, qp, arg, last[k] if warm else None)
        alone.append((sol, st))
        last[k] = sol
    # in the mix: all requests through the server, small lanes so that
    # micro-batches of different requests run concurrently
    src = QpBatch([qp for _, qp, _ in reqs], device=None)
    with server.Server(1 << 30, lanes=3, max_batch=5, arg=arg) as srv:
        tickets = [srv.submit(src, i, key=k + 1, warm=w) for i, (k, _, w) in enumerate(reqs)]
        srv.drain(120.0)
        rep = srv.report()
        results = [srv.result(t) for t in tickets]
    assert rep["completed"] == len(reqs) and rep["rejected"] == 0 and rep["failed"] == 0
    assert rep["warm_hits"] == sum(w for _, _, w in reqs) and rep["warm_misses"] == 0
    assert rep["batches"] >= len(reqs) // 5
    bad = []
    for i, ((k, qp, warm), (info, sol)) in enumerate(zip(reqs, results)):
        (ya, pia, lama, ta), st = alone[i]
        assert info.code == 0 and info.done == 1
        assert info.warm_used == int(warm)
        assert info.latency_ns >= info.wait_ns >= 0
        same = all(np.array_equal(a, b) for a, b in zip(sol, (ya, pia, lama, ta)))
        if not (same and info.stats.iters == st.iters and info.stats.status == st.status == 0):
            bad.append((i, k, warm, info.stats.status, st.status, info.stats.iters, st.iters,
                        info.stats.flags, st.flags, float(np.max(np.abs(sol[0] - ya)))))
    assert not bad, "requests differing from their solve alone (i, key, warm, status, iters, flags, dy): %s" % bad
    # the oracle on cold requests: KKT residuals at the exit rule, the
    # solution of the oracle run with the same exit rule, and (when the tight
    # oracle converges) the exact solution within the degenerate-bound bound
    for i in (0, 3, len(reqs) // 3 - 1):
        k, qp, warm = reqs[i]
        assert not warm
        same, tight = GP.oracle_pair(qp)
        info, (y, pi, lam, t) = results[i]
        kkt = O.full_residuals(qp, y, pi, lam, t)
        assert max(kkt[:4]) <= GP.KKT_TOL * 1.01, (i, kkt)
        assert same.status == O.CONVERGED
        assert GP.rel_err(y, same.y) <= SOL_TOL, (i, GP.rel_err(y, same.y))
        if tight.status == O.CONVERGED:
            assert GP.rel_err(y, tight.y) <= EXACT_TOL, (i, GP.rel_err(y, tight.y))


def test_warm_repeats_take_fewer_iterations(env):
    gq, server, QpBatch, torch = env
    reqs = request_stream(nkeys=10, nrep=1, seed=1)
    src = QpBatch([qp for _, qp, _ in reqs], device=None)
    with server.Server(1 << 30, lanes=2, max_batch=8) as srv:
        tickets = [srv.submit(src, i, key=k + 1, warm=w) for i, (k, _, w) in enumerate(reqs)]
        srv.drain(120.0)
        infos = [srv.result(t)[0] for t in tickets]
    cold = [inf.stats.iters for inf, (_, _, w) in zip(infos, reqs) if not w]
    warm = [inf.stats.iters for inf, (_, _, w) in zip(infos, reqs) if w]
    assert all(inf.stats.status == gq.STATUS_CONVERGED for inf in infos)
    assert np.mean(warm) < np.mean(cold), (cold, warm)


def test_admission_by_device_budget(env):
    """Micro-batches are split to fit a lane's share of the arena, and a QP
    larger than a whole share is rejected with GQ_ERR_SIZE while the rest
    complete."""
    gq, server, QpBatch, torch = env
    small = [W.small_random_qp(i) for i in range(12)]
    big = W.ragged_random_qp(0, N_range=(100, 100), nx_range=(64, 64))
    one_small = QpBatch(small[:1], device=None).sizes
    one_big = QpBatch([big], device=None).sizes
    need_small = sum(((x + 255) // 256) * 256 for x in (one_small.in_bytes, one_small.sol_bytes, one_small.ws_bytes))
    need_big = one_big.in_bytes + one_big.sol_bytes + one_big.ws_bytes
    lane = 3 * need_small + 8192          # room for about three small QPs per micro-batch
    assert lane < need_big
    src = QpBatch(small + [big], device=None)
    budget = 2 * lane
    with server.Server(budget, lanes=2, max_batch=64, cache_bytes=0, pinned_bytes=budget) as srv:
        tickets = [srv.submit(src, i) for i in range(len(small) + 1)]
        srv.drain(60.0)
        rep = srv.report()
        infos = [srv.result(t)[0] for t in tickets]
    assert infos[-1].code == gq.GQ_ERR_SIZE
    assert all(inf.code == 0 and inf.stats.status == gq.STATUS_CONVERGED for inf in infos[:-1])
    assert max(inf.batch_size for inf in infos[:-1]) <= 4
    assert rep["rejected"] == 1 and rep["completed"] == len(small)
    assert rep["batches"] >= len(small) // 4


def test_lanes_overlap_and_keys_stay_ordered(env):
    gq, server, QpBatch, torch = env
    qps = [W.ragged_random_qp(i) for i in range(24)]
    src = QpBatch(qps, device=None)
    with server.Server(1 << 30, lanes=4, max_batch=2) as srv:
        # every QP twice under the same key: the second waits for the first
        arrivals, tickets = [], []
        for rnd in range(2):
            for i in range(24):
                t = server.now_ns()
                arrivals.append(t)
                tickets.append(srv.submit(src, i, key=i + 1, warm=rnd == 1, t_arrival_ns=t))
        srv.drain(120.0)
        rep = srv.report()
        infos = [srv.result(t)[0] for t in tickets]
    assert rep["max_lanes_busy"] >= 2          # micro-batches ran concurrently
    assert rep["completed"] == 48 and rep["warm_hits"] == 24
    for i in range(24):
        first, second = infos[i], infos[24 + i]
        assert first.stats.status == second.stats.status == gq.STATUS_CONVERGED
        assert second.warm_used == 1
        # the repeat was admitted only after the first solve of its key was
        # visible on the host
        assert arrivals[24 + i] + second.wait_ns >= arrivals[i] + first.latency_ns
        assert second.stats.iters <= first.stats.iters


@pytest.mark.parametrize("class_ratio", [4.0, 1.0])
def test_size_classes_group_micro_batches(env, class_ratio):
    """With size classes a micro-batch takes only requests of the oldest
    eligible request's cost class, so small QPs never share a batch (and its
    completion time) with large ones; class_ratio <= 1 turns this off."""
    gq, server, QpBatch, torch = env
    small = [W.small_random_qp(i) for i in range(6)]
    big = [W.large_stage_qp(i, N=4) for i in range(3)]
    qps = [q for pair in zip(small, big + [None] * 3) for q in pair if q is not None]
    src = QpBatch(qps, device=None)
    is_big = [any(q is b for b in big) for q in qps]
    with server.Server(1 << 30, lanes=1, max_batch=1000, max_wait_us=200000, class_ratio=class_ratio) as srv:
        tickets = [srv.submit(src, i) for i in range(len(qps))]
        srv.drain(120.0)
        infos = [srv.result(t)[0] for t in tickets]
    assert all(inf.code == 0 and inf.stats.status == gq.STATUS_CONVERGED for inf in infos)
    sizes = [inf.batch_size for inf in infos]
    if class_ratio > 1.0:
        assert all(sz == (3 if b else 6) for sz, b in zip(sizes, is_big)), sizes
    else:
        assert all(sz == 9 for sz in sizes), sizes



def test_bad_requests_and_shutdown_fail_cleanly(env):
    """A request for a QP index outside its source is refused at submit, and
    destroying a server with requests still queued returns promptly (the
    micro-batch in flight finishes, the rest are dropped) and leaves the GPU
    usable."""
    import time
    gq, server, QpBatch, torch = env
    qps = [W.ragged_random_qp(i) for i in range(6)]
    src = QpBatch(qps, device=None)
    srv = server.Server(1 << 28, lanes=1, max_batch=1, max_wait_us=0)
    with pytest.raises(gq.GqError) as e:
        srv.submit(src, 17)
    assert e.value.code == gq.GQ_ERR_ARG
    for i in range(6):
        srv.submit(src, i)
    t0 = time.monotonic()
    srv.close()
    assert time.monotonic() - t0 < 30.0
    b = QpBatch([W.small_random_qp(0)])
    b.upload()
    b.solve(gq.default_arg(0, 1))
    b.download()
    torch.cuda.synchronize()
    assert b.all_stats()["status"][0] == gq.STATUS_CONVERGED
