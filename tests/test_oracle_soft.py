"""Pins of the oracle's soft constraints (Sec. 2.2: slack variables with
diagonal L2 and linear L1 costs that relax box and general constraints).

Each check fixes the soft solution by something other than the oracle's own
assembly of the slacks:
* a scalar problem whose soft optimum has a closed form (Z, z, both sides);
* exact-penalty theory: with Z = 0 and z above the hard multipliers the soft
  problem has the hard problem's solution and zero slacks;
* brute force over active sets of the soft problem written out here, from
  the condensed QP with explicit slack columns, on tiny instances including
  ones whose hard version is infeasible.
"""
import itertools

import numpy as np
import pytest

from oracle import ocp_ipm as O
from paper_2003_02547_gb300 import workloads as W
from test_oracle_pins import condensed, random_lq

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def scalar_qp(x0, lo, hi, q=1.0, r=1.0):
    """N = 1, nx_0 = 0, nu_0 = 1: x_1 = x0 + u_0, cost 1/2 r u^2 + 1/2 q x_1^2,
    box lo <= x_1 <= hi on stage 1."""
    A = np.eye(1)
    B = np.eye(1)
    qp = W._assemble(1, A, B, np.zeros(1), q * np.eye(1), r * np.eye(1), np.zeros((1, 1)),
                     np.zeros(1), np.zeros(1), np.array([x0]), ubound=np.inf, xbound=1.0, name="scalar")
    qp.lbx[1] = np.array([lo])
    qp.ubx[1] = np.array([hi])
    qp.idxbu[0] = np.zeros(0, dtype=int)
    qp.lbu[0] = np.zeros(0)
    qp.ubu[0] = np.zeros(0)
    qp.validate()
    return qp


@pytest.mark.parametrize("side", ["lower", "upper"])
@pytest.mark.parametrize("Z,z", [(4.0, 0.5), (0.7, 0.0), (10.0, 2.0)])
def test_scalar_soft_bound_closed_form(side, Z, z):
    """Stationarity of 1/2 r u^2 + 1/2 q (x0+u)^2 + 1/2 Z s^2 + z s with the
    relaxed side active, s = lo - x0 - u > 0 (lower) or s = x0 + u - hi > 0
    (upper): u = (Z (lo - x0) + z - q x0) / (r + q + Z) for the lower side and
    u = (Z (hi - x0) - z - q x0) / (r + q + Z) for the upper side."""
    q, r = 1.0, 0.5
    if side == "lower":
        x0, lo, hi = -3.0, 1.0, 5.0
        u = (Z * (lo - x0) + z - q * x0) / (r + q + Z)
        s = lo - x0 - u
    else:
        x0, lo, hi = 3.0, -5.0, -1.0
        u = (Z * (hi - x0) - z - q * x0) / (r + q + Z)
        s = x0 + u - hi
    assert s > 0
    qp = W.soften(scalar_qp(x0, lo, hi, q, r), [1], "x", Z=Z, z=z, ls=0.0)
    res = O.solve(qp)
    assert res.status == O.CONVERGED
    st = O.split_stages(qp, res.dq, res.y)
    sl = O.split_slacks(qp, res.dq, res.y)[1]
    np.testing.assert_allclose(st[0][0], [u], atol=1e-9)
    np.testing.assert_allclose(st[1][1], [x0 + u], atol=1e-9)
    relaxed, other = (sl[0], sl[1]) if side == "lower" else (sl[1], sl[0])
    np.testing.assert_allclose(relaxed, [s], atol=1e-9)
    # the other slack's bound is active at 0; with z = 0 its multiplier is 0
    # too (degenerate), and an IPM reaches such a bound only to about
    # sqrt(mu) ~ 1e-5 at the 1e-10 exit
    np.testing.assert_allclose(other, [0.0], atol=1e-4 if z == 0.0 else 1e-8)


def test_scalar_soft_bound_inactive_when_feasible():
    """The relaxed bound is not reached: slacks 0 and the unconstrained LQR
    optimum u = -q x0 / (r + q)."""
    q, r, x0 = 1.0, 0.5, 0.4
    qp = W.soften(scalar_qp(x0, -2.0, 2.0, q, r), [1], "x", Z=1.0, z=1.0)
    res = O.solve(qp)
    assert res.status == O.CONVERGED
    st = O.split_stages(qp, res.dq, res.y)
    np.testing.assert_allclose(st[0][0], [-q * x0 / (r + q)], atol=1e-9)
    np.testing.assert_allclose(np.concatenate(O.split_slacks(qp, res.dq, res.y)[1]), 0.0, atol=1e-8)


@pytest.mark.parametrize("which", ["x", "u", "all"])
def test_exact_l1_penalty_recovers_hard_solution(which):
    """Exact penalty (Nocedal & Wright, Thm. 17.3): with Z = 0 and z larger
    than every hard multiplier the soft problem's minimiser is the hard one,
    with zero slacks."""
    qp = W.small_random_qp(3, x0_scale=2.0)
    hard = O.solve(qp)
    assert hard.status == O.CONVERGED
    lam_max = float(np.max(hard.lam))
    assert lam_max > 1e-3    # some constraint is active
    soft = W.soften(qp, range(qp.N + 1), which, Z=0.0, z=10.0 * lam_max + 1.0)
    res = O.solve(soft)
    assert res.status == O.CONVERGED
    a = O.split_stages(qp, hard.dq, hard.y)
    b = O.split_stages(soft, res.dq, res.y)
    for n in range(qp.N + 1):
        np.testing.assert_allclose(b[n][0], a[n][0], atol=1e-7)
        np.testing.assert_allclose(b[n][1], a[n][1], atol=1e-7)
    for sl, su in O.split_slacks(soft, res.dq, res.y):
        assert np.all(np.abs(sl) <= 1e-7) and np.all(np.abs(su) <= 1e-7)


def test_small_l1_penalty_changes_solution():
    """The converse: a penalty below the hard multiplier lets the slack open
    (the soft optimum differs from the hard one)."""
    qp = W.small_random_qp(3, x0_scale=2.0)
    hard = O.solve(qp)
    soft = W.soften(qp, range(qp.N + 1), "all", Z=0.0, z=1e-3 * float(np.max(hard.lam)))
    res = O.solve(soft)
    assert res.status == O.CONVERGED
    slk = np.concatenate([np.concatenate(p) for p in O.split_slacks(soft, res.dq, res.y)])
    assert np.max(slk) > 1e-3


# ----------------------------------------------------------------------------
# brute force over active sets of the soft problem
# ----------------------------------------------------------------------------
def soft_rows(qp):
    """The soft QP in w = [z; s] (z the condensed decision vector, s all slacks
    stage by stage as [s^l; s^u]): cost 1/2 w'Hw w + hw'w and one-sided or
    two-sided rows lo <= G w <= hi, written from the problem statement."""
    Hz, hz, G, lo, hi, Umap, Xmap, xoff = condensed(qp)
    nz = Hz.shape[0]
    ns = [qp.ns(n) for n in range(qp.N + 1)]
    nsl = 2 * sum(ns)
    H = np.zeros((nz + nsl, nz + nsl))
    H[:nz, :nz] = Hz
    h = np.concatenate([hz, np.zeros(nsl)])
    rows, rlo, rhi = [], [], []
    # constraint rows of each stage start at this offset in G
    base = np.cumsum([0] + [qp.nbu(n) + qp.nbx(n) + qp.ng(n) for n in range(qp.N + 1)])
    soft_of = {}
    col = nz
    for n in range(qp.N + 1):
        for k in range(ns[n]):
            jl, ju = col + k, col + ns[n] + k
            H[jl, jl], H[ju, ju] = qp.Zl[n][k], qp.Zu[n][k]
            h[jl], h[ju] = qp.zl[n][k], qp.zu[n][k]
            soft_of[base[n] + int(qp.idxs[n][k])] = (jl, ju)
            for j, bnd in ((jl, qp.lls[n][k]), (ju, qp.lus[n][k])):
                e = np.zeros(nz + nsl)
                e[j] = 1.0
                rows.append(e)
                rlo.append(bnd)
                rhi.append(np.inf)
        col += 2 * ns[n]
    for i in range(G.shape[0]):
        g = np.concatenate([G[i], np.zeros(nsl)])
        if i in soft_of:
            jl, ju = soft_of[i]
            gl = g.copy()
            gl[jl] = 1.0           # c + s^l >= lo
            gu = g.copy()
            gu[ju] = -1.0          # c - s^u <= hi
            rows += [gl, gu]
            rlo += [lo[i], -np.inf]
            rhi += [np.inf, hi[i]]
        else:
            rows.append(g)
            rlo.append(lo[i])
            rhi.append(hi[i])
    return H, h, np.array(rows), np.array(rlo), np.array(rhi), Umap, Xmap, xoff, nz


def brute_force_rows(H, h, G, lo, hi):
    """Every KKT point of min 1/2 w'Hw + h'w s.t. lo <= Gw <= hi by
    enumerating, per row, the finite bounds it may be active at."""
    m, nw = G.shape
    opts = [[0] + ([1] if np.isfinite(lo[i]) else []) + ([2] if np.isfinite(hi[i]) else []) for i in range(m)]
    found = []
    for act in itertools.product(*opts):
        idx = [i for i in range(m) if act[i]]
        if len(idx) > nw:
            continue
        Ga = G[idx] if idx else np.zeros((0, nw))
        if idx and np.linalg.matrix_rank(Ga) < len(idx):
            continue
        rb = [lo[i] if act[i] == 1 else hi[i] for i in idx]
        K = np.block([[H, Ga.T], [Ga, np.zeros((len(idx), len(idx)))]])
        try:
            sol = np.linalg.solve(K, np.concatenate([-h, rb]))
        except np.linalg.LinAlgError:
            continue
        w = sol[:nw]
        mult = -sol[nw:]
        gw = G @ w
        if np.any(gw < lo - 1e-9) or np.any(gw > hi + 1e-9):
            continue
        if any((act[i] == 1 and mult[j] < -1e-9) or (act[i] == 2 and mult[j] > 1e-9) for j, i in enumerate(idx)):
            continue
        found.append(w)
    return found


def tiny_soft(seed):
    rng = np.random.default_rng([11, seed])
    qp = random_lq(200 + seed, N=2, nxs=[0, 2, 2], nus=[1, 1, 0], boxes=True, tight=0.4)
    qp.idxbx[2] = qp.idxbx[2][:1]
    qp.lbx[2] = qp.lbx[2][:1]
    qp.ubx[2] = qp.ubx[2][:1]
    qp.C[1] = rng.standard_normal((1, 2))
    qp.D[1] = rng.standard_normal((1, 1))
    qp.lg[1] = np.array([-0.2])
    qp.ug[1] = np.array([0.1])
    qp.validate()
    Z = float(rng.uniform(0.2, 3.0)) if seed % 3 else 0.0
    z = float(rng.uniform(0.05, 1.0))
    # soft: the general row of stage 1 and the state box of stage 2
    g1 = W.soften(qp, [1], "g", Z=Z, z=z, ls=0.0)
    x2 = W.soften(qp, [2], "x", Z=Z, z=z, ls=float(rng.uniform(-0.1, 0.0)))
    for f in ("idxs", "Zl", "Zu", "zl", "zu", "lls", "lus"):
        getattr(g1, f)[2] = getattr(x2, f)[2]
    g1.validate()
    return g1


SOFT_SEEDS = range(16)


@pytest.mark.parametrize("seed", SOFT_SEEDS)
def test_soft_brute_force_active_sets(seed):
    """Tiny soft QPs (N = 2; the general row of stage 1 and the state box of
    stage 2 soft, the latter with negative slack bounds; tight boxes so that
    slacks open): the unique KKT point found by enumeration equals the
    oracle's solution, slacks included."""
    qp = tiny_soft(seed)
    H, h, G, lo, hi, Umap, Xmap, xoff, nz = soft_rows(qp)
    found = brute_force_rows(H, h, G, lo, hi)
    res = O.solve(qp)
    if not found:
        # the hard boxes that remain admit no point: no KKT point exists
        assert res.status != O.CONVERGED
        return
    w = found[0]
    if H[nz:, nz:].diagonal().min() > 0:   # strictly convex: one KKT point
        for w2 in found[1:]:
            np.testing.assert_allclose(w2, w, atol=1e-8)
    assert res.status == O.CONVERGED
    st = O.split_stages(qp, res.dq, res.y)
    if H[nz:, nz:].diagonal().min() > 0:
        # 1e-6: a slack resting on its bound with a zero multiplier
        # (degenerate) is reached only to about sqrt(mu) by an IPM; a wrong
        # sign or a dropped slack term moves the solution by O(0.1)
        for n in range(qp.N + 1):
            np.testing.assert_allclose(st[n][0], Umap[n] @ w[:nz], atol=1e-6)
            np.testing.assert_allclose(st[n][1], Xmap[n] @ w[:nz] + xoff[n], atol=1e-6)
        s_or = np.concatenate([np.concatenate(p) for p in O.split_slacks(qp, res.dq, res.y)])
        np.testing.assert_allclose(s_or, w[nz:], atol=1e-6)
    # the optimal value agrees in every case (slacks with only a linear cost
    # may have several minimisers): the oracle's point, written as w, is
    # feasible for the rows above and has the enumerated point's cost
    z_or = np.concatenate([st[0][1]] + [st[n][0] for n in range(qp.N + 1)])
    s_or = np.concatenate([np.concatenate(p) for p in O.split_slacks(qp, res.dq, res.y)])
    w_or = np.concatenate([z_or, s_or])
    gw = G @ w_or
    assert np.all(gw >= lo - 1e-8) and np.all(gw <= hi + 1e-8)
    f = lambda v: 0.5 * v @ H @ v + h @ v
    assert abs(f(w_or) - f(w)) <= 1e-8 * max(1.0, abs(f(w)))


def test_soft_brute_force_instances_engage_slacks():
    """The instances above are not vacuous: most have a KKT point, and in
    most of those some slack is open at the optimum."""
    feasible = opened = 0
    for seed in SOFT_SEEDS:
        qp = tiny_soft(seed)
        H, h, G, lo, hi, *_, nz = soft_rows(qp)
        found = brute_force_rows(H, h, G, lo, hi)
        if found:
            feasible += 1
            opened += int(np.max(np.abs(found[0][nz:] - np.concatenate(
                [np.concatenate([qp.lls[n], qp.lus[n]]) for n in range(qp.N + 1)]))) > 1e-6)
    assert feasible >= len(SOFT_SEEDS) // 2 and opened >= feasible // 2, (feasible, opened)


def test_soft_problem_with_infeasible_hard_version():
    """Hard bounds that no input can meet (|x_1| <= 0.01 against a large x0)
    have no KKT point; relaxed, the oracle converges and the slacks carry the
    violation."""
    qp = W.small_random_qp(5, x0_scale=2.0)
    qp.lbx[1] = np.full_like(qp.lbx[1], -0.01)
    qp.ubx[1] = np.full_like(qp.ubx[1], 0.01)
    qp.lbu[0] = np.full_like(qp.lbu[0], -0.01)
    qp.ubu[0] = np.full_like(qp.ubu[0], 0.01)
    qp.validate()
    assert O.solve(qp).status != O.CONVERGED
    soft = W.soften(qp, [1], "x", Z=1.0, z=0.1)
    res = O.solve(soft)
    assert res.status == O.CONVERGED
    sl, su = O.split_slacks(soft, res.dq, res.y)[1]
    x1 = O.split_stages(soft, res.dq, res.y)[1][1]
    viol = np.maximum(qp.lbx[1] - x1[qp.idxbx[1]], 0.0) + np.maximum(x1[qp.idxbx[1]] - qp.ubx[1], 0.0)
    assert np.max(viol) > 0.1
    np.testing.assert_allclose(sl + su, viol, atol=1e-8)
