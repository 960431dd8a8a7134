"""Pins of the CPU oracle to results fixed by mathematics, not by the oracle.

Each pin reaches the QP solution by a different method than the oracle's
dense reduced-KKT IPM:

* the classical (not square-root) Riccati difference equation written here
  from dynamic programming, for unconstrained LQ problems;
* the infinite-horizon limit, scipy.linalg.solve_discrete_are;
* enumeration of all active sets of the condensed (states eliminated) QP;
* the unreduced Newton system of eq. (delta) solved in one piece;
* invariants: zero duality gap, symmetry under x0 -> -x0, dense vs sparse.

The paper prints no solution values (Table 1 holds timings only), so there
is no printed worked example to pin against.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg

from oracle import ocp_ipm as O
from paper_2003_02547_gb300 import workloads as W


# ----------------------------------------------------------------------------
# random stage-varying OCP QPs (independent of the workload generators)
# ----------------------------------------------------------------------------
def random_lq(seed, N=5, nxs=None, nus=None, boxes=False, ng=0, tight=1.0):
    rng = np.random.default_rng([99, seed])
    if nxs is None:
        nxs = [int(rng.integers(1, 5)) for _ in range(N + 1)]
    if nus is None:
        nus = [int(rng.integers(1, 4)) for _ in range(N + 1)]
        nus[N] = int(rng.integers(0, 2))
    A, B, b = [], [], []
    for n in range(N):
        A.append(rng.standard_normal((nxs[n + 1], nxs[n])) * 0.7)
        B.append(rng.standard_normal((nxs[n + 1], nus[n])))
        b.append(rng.standard_normal(nxs[n + 1]) * 0.3)
    Q, S, R, q, r = [], [], [], [], []
    for n in range(N + 1):
        nx, nu = nxs[n], nus[n]
        # a random positive definite stage Hessian [[R, S], [S', Q]]
        G = rng.standard_normal((nx + nu, nx + nu))
        Hn = G @ G.T + 0.5 * np.eye(nx + nu)
        R.append(Hn[:nu, :nu].copy())
        S.append(Hn[:nu, nu:].copy())
        Q.append(Hn[nu:, nu:].copy())
        q.append(rng.standard_normal(nx))
        r.append(rng.standard_normal(nu))
    ibu, lbu, ubu, ibx, lbx, ubx, C, D, lg, ug = ([] for _ in range(10))
    for n in range(N + 1):
        nx, nu = nxs[n], nus[n]
        if boxes:
            iu = np.arange(nu, dtype=np.int64)
            ix = np.arange(nx, dtype=np.int64)
            ibu.append(iu)
            lbu.append(-tight * rng.uniform(0.2, 1.0, nu))
            ubu.append(tight * rng.uniform(0.2, 1.0, nu))
            ibx.append(ix)
            lbx.append(-tight * rng.uniform(0.5, 2.0, nx))
            ubx.append(tight * rng.uniform(0.5, 2.0, nx))
        else:
            for L in (ibu, ibx):
                L.append(np.zeros(0, dtype=np.int64))
            for L in (lbu, ubu, lbx, ubx):
                L.append(np.zeros(0))
        C.append(rng.standard_normal((ng, nx)))
        D.append(rng.standard_normal((ng, nu)))
        lg.append(-tight * rng.uniform(0.5, 1.5, ng))
        ug.append(tight * rng.uniform(0.5, 1.5, ng))
    qp = W.OcpQp(N=N, nx=nxs, nu=nus, A=A, B=B, b=b, Q=Q, S=S, R=R, q=q, r=r,
                 idxbu=ibu, lbu=lbu, ubu=ubu, idxbx=ibx, lbx=lbx, ubx=ubx,
                 C=C, D=D, lg=lg, ug=ug, name=f"rand{seed}")
    qp.validate()
    return qp


def riccati_dp(qp):
    """Classical Riccati difference equation by dynamic programming.

    V_N = stage-N cost minimised over u_N; V_n(x) = min_u l_n(u, x) +
    V_{n+1}(A x + B u + b) with V(x) = 1/2 x'Px + p'x.  Returns per-stage
    (u_n, x_n) and the cost-to-go gradients pi_{n+1} = P_{n+1} x_{n+1} + p_{n+1}.
    """
    N = qp.N
    P = [None] * (N + 1)
    p = [None] * (N + 1)
    K = [None] * (N + 1)
    k = [None] * (N + 1)
    for n in range(N, -1, -1):
        Qb, Sb, Rb = qp.Q[n].copy(), qp.S[n].copy(), qp.R[n].copy()
        qb, rb = qp.q[n].copy(), qp.r[n].copy()
        if n < N:
            An, Bn, bn = qp.A[n], qp.B[n], qp.b[n]
            Pn1, pn1 = P[n + 1], p[n + 1]
            Qb += An.T @ Pn1 @ An
            Sb += Bn.T @ Pn1 @ An
            Rb += Bn.T @ Pn1 @ Bn
            w = Pn1 @ bn + pn1
            qb += An.T @ w
            rb += Bn.T @ w
        if Rb.size:
            K[n] = -np.linalg.solve(Rb, Sb)
            k[n] = -np.linalg.solve(Rb, rb)
            P[n] = Qb + Sb.T @ K[n]
            p[n] = qb + Sb.T @ k[n]
        else:
            K[n] = np.zeros((0, Qb.shape[0]))
            k[n] = np.zeros(0)
            P[n], p[n] = Qb, qb
    xs, us, pis = [], [], []
    x = -np.linalg.solve(P[0], p[0]) if qp.nx[0] else np.zeros(0)
    for n in range(N + 1):
        u = K[n] @ x + k[n]
        xs.append(x)
        us.append(u)
        if n < N:
            x = qp.A[n] @ x + qp.B[n] @ u + qp.b[n]
            pis.append(P[n + 1] @ x + p[n + 1])
    return us, xs, pis


def test_unconstrained_matches_riccati_dp():
    """P1: with no inequalities the IPM reduces to one KKT solve, whose
    result must equal the classical Riccati recursion (stage-varying sizes,
    non-zero S, q, r, b)."""
    for seed in range(6):
        qp = random_lq(seed, N=6)
        res = O.solve(qp)
        assert res.status == O.CONVERGED
        us, xs, pis = riccati_dp(qp)
        st = O.split_stages(qp, res.dq, res.y)
        for n in range(qp.N + 1):
            np.testing.assert_allclose(st[n][0], us[n], rtol=1e-9, atol=1e-10)
            np.testing.assert_allclose(st[n][1], xs[n], rtol=1e-9, atol=1e-10)
        pi_ref = np.concatenate(pis)
        np.testing.assert_allclose(res.pi, pi_ref, rtol=1e-9, atol=1e-10)


def test_long_horizon_matches_dare():
    """P1 limit: for a long horizon the first feedback of the time-invariant
    LQR equals the infinite-horizon gain from scipy's DARE solver."""
    qp0 = W.small_random_qp(3, N=200, x0_scale=1e-3)
    # drop the boxes: an unconstrained problem
    qp = W.small_random_qp(3, N=200, x0_scale=1e-3)
    for n in range(qp.N + 1):
        qp.idxbu[n] = np.zeros(0, dtype=np.int64)
        qp.idxbx[n] = np.zeros(0, dtype=np.int64)
        qp.lbu[n] = qp.ubu[n] = qp.lbx[n] = qp.ubx[n] = np.zeros(0)
    res = O.solve(qp)
    assert res.status == O.CONVERGED
    A, B = qp0.A[1], qp0.B[1]
    Q, R = np.eye(4), 0.1 * np.eye(2)
    P = scipy.linalg.solve_discrete_are(A, B, Q, R)
    Kinf = -np.linalg.solve(R + B.T @ P @ B, B.T @ P @ A)
    u0 = res.y[:2]
    np.testing.assert_allclose(u0, Kinf @ qp.x0, rtol=1e-8, atol=1e-14)


def test_inactive_boxes_equal_lqr():
    """P2: the small workload with x0 scaled by 1e-3 leaves every box
    inactive, so the IPM solution equals the unconstrained LQR."""
    qp = W.small_random_qp(0, x0_scale=1e-3)
    res = O.solve(qp)
    assert res.status == O.CONVERGED
    us, xs, _ = riccati_dp(qp)
    st = O.split_stages(qp, res.dq, res.y)
    for n in range(qp.N + 1):
        np.testing.assert_allclose(st[n][0], us[n], rtol=1e-7, atol=1e-11)
        np.testing.assert_allclose(st[n][1], xs[n], rtol=1e-7, atol=1e-11)


# ----------------------------------------------------------------------------
# brute force over active sets of the condensed QP
# ----------------------------------------------------------------------------
def condensed(qp):
    """Eliminate the states: x_n = T_n z + t_n with z = [x_0; u_0; ...; u_N].
    Returns the QP in z: cost 1/2 z'Hz z + hz'z, constraint rows G z in [lo, hi]."""
    N = qp.N
    nz = qp.nx[0] + sum(qp.nu)
    # affine maps for x_n and u_n in terms of z
    uo = np.cumsum([qp.nx[0]] + list(qp.nu))
    Xmap, xoff = [], []
    Tx = np.zeros((qp.nx[0], nz))
    Tx[:, :qp.nx[0]] = np.eye(qp.nx[0])
    tx = np.zeros(qp.nx[0])
    Umap = []
    for n in range(N + 1):
        Tu = np.zeros((qp.nu[n], nz))
        Tu[:, uo[n]:uo[n] + qp.nu[n]] = np.eye(qp.nu[n])
        Umap.append(Tu)
        Xmap.append(Tx)
        xoff.append(tx)
        if n < N:
            Tx = qp.A[n] @ Tx + qp.B[n] @ Tu
            tx = qp.A[n] @ tx + qp.b[n]
    Hz = np.zeros((nz, nz))
    hz = np.zeros(nz)
    G, lo, hi = [], [], []
    for n in range(N + 1):
        Tu, Tx, tx = Umap[n], Xmap[n], xoff[n]
        # cost 1/2 u'Ru + u'S x + 1/2 x'Qx + r'u + q'x, x = Tx z + tx
        Hz += Tu.T @ qp.R[n] @ Tu + Tu.T @ qp.S[n] @ Tx + Tx.T @ qp.S[n].T @ Tu + Tx.T @ qp.Q[n] @ Tx
        hz += Tu.T @ (qp.r[n] + qp.S[n] @ tx) + Tx.T @ (qp.q[n] + qp.Q[n] @ tx)
        for kk, i in enumerate(qp.idxbu[n]):
            G.append(Tu[int(i)])
            lo.append(qp.lbu[n][kk])
            hi.append(qp.ubu[n][kk])
        for kk, i in enumerate(qp.idxbx[n]):
            G.append(Tx[int(i)])
            lo.append(qp.lbx[n][kk] - tx[int(i)])
            hi.append(qp.ubx[n][kk] - tx[int(i)])
        for kk in range(qp.ng(n)):
            row = qp.D[n][kk] @ Tu + qp.C[n][kk] @ Tx
            G.append(row)
            off = qp.C[n][kk] @ tx
            lo.append(qp.lg[n][kk] - off)
            hi.append(qp.ug[n][kk] - off)
    return Hz, hz, np.array(G), np.array(lo), np.array(hi), Umap, Xmap, xoff


def brute_force(qp):
    """Enumerate every active set (each constraint free, at its lower or at
    its upper bound), solve the equality-constrained QP, keep the one that is
    primal feasible with correctly signed multipliers."""
    Hz, hz, G, lo, hi, Umap, Xmap, xoff = condensed(qp)
    m = G.shape[0]
    nz = Hz.shape[0]
    best = []
    for act in itertools.product((0, 1, 2), repeat=m):
        idx = [i for i in range(m) if act[i]]
        rhs_b = [lo[i] if act[i] == 1 else hi[i] for i in idx]
        if any(not np.isfinite(v) for v in rhs_b):
            continue
        Ga = G[idx] if idx else np.zeros((0, nz))
        if len(idx) > nz or (idx and np.linalg.matrix_rank(Ga) < len(idx)):
            continue   # dependent active rows: not a vertex of this QP
        K = np.block([[Hz, Ga.T], [Ga, np.zeros((len(idx), len(idx)))]])
        rhs = np.concatenate([-hz, rhs_b])
        try:
            sol = np.linalg.solve(K, rhs)
        except np.linalg.LinAlgError:
            continue
        z = sol[:nz]
        nu_ = -sol[nz:]          # H z + h = Ga' nu_  ->  nu_ = multipliers
        cz = G @ z
        if np.any(cz < lo - 1e-9) or np.any(cz > hi + 1e-9):
            continue
        ok = True
        for j, i in enumerate(idx):
            # lower active: multiplier of (Gz - lo >= 0) must be >= 0
            if act[i] == 1 and nu_[j] < -1e-9:
                ok = False
            if act[i] == 2 and nu_[j] > 1e-9:
                ok = False
        if ok:
            best.append(z)
    if not best:
        return None
    z = best[0]
    for z2 in best[1:]:
        assert np.allclose(z, z2, atol=1e-8)
    us = [Umap[n] @ z for n in range(qp.N + 1)]
    xs = [Xmap[n] @ z + xoff[n] for n in range(qp.N + 1)]
    return us, xs


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_active_sets(seed):
    """P3: tiny QPs (N = 2, x_0 eliminated, 6 two-sided constraints incl. one
    general row), 3^6 active sets, unique KKT point == IPM solution.  Draws
    without any KKT point are infeasible: the IPM must not report success."""
    rng = np.random.default_rng([7, seed])
    nxs, nus = [0, 2, 2], [1, 1, 0]
    qp = random_lq(100 + seed, N=2, nxs=nxs, nus=nus, boxes=True, tight=0.35)
    # keep 5 boxes and one general constraint at stage 1
    qp.idxbx[2] = qp.idxbx[2][:1]
    qp.lbx[2] = qp.lbx[2][:1]
    qp.ubx[2] = qp.ubx[2][:1]
    qp.C[1] = rng.standard_normal((1, 2))
    qp.D[1] = rng.standard_normal((1, 1))
    qp.lg[1] = np.array([-0.3])
    qp.ug[1] = np.array([0.4])
    qp.validate()
    res = O.solve(qp)
    bf = brute_force(qp)
    if bf is None:
        assert res.status != O.CONVERGED
        return
    assert res.status == O.CONVERGED
    us, xs = bf
    st = O.split_stages(qp, res.dq, res.y)
    for n in range(qp.N + 1):
        np.testing.assert_allclose(st[n][0], us[n], atol=1e-9)
        np.testing.assert_allclose(st[n][1], xs[n], atol=1e-9)


def test_brute_force_with_free_initial_state_and_masks():
    """P3 variant: nx_0 > 0 (x_0 free, boxed) and one-sided (masked) bounds."""
    qp = random_lq(555, N=2, nxs=[1, 2, 1], nus=[1, 1, 0], boxes=True, tight=0.3)
    qp.lbu[1] = np.array([-np.inf])
    qp.ubx[1] = np.array([np.inf, qp.ubx[1][1]])
    qp.validate()
    res = O.solve(qp)
    assert res.status == O.CONVERGED
    us, xs = brute_force(qp)
    st = O.split_stages(qp, res.dq, res.y)
    for n in range(qp.N + 1):
        np.testing.assert_allclose(st[n][0], us[n], atol=1e-9)
        np.testing.assert_allclose(st[n][1], xs[n], atol=1e-9)
    # masked sides report lambda = 0
    assert np.all(res.lam[~res.dq.active] == 0.0)


# ----------------------------------------------------------------------------
# Newton step: reduced system (Sec. 3.3) == unreduced system (eq. delta)
# ----------------------------------------------------------------------------
def test_reduced_newton_step_equals_full_system():
    for seed in range(4):
        qp = random_lq(200 + seed, N=4, boxes=True, ng=2)
        dq = O.assemble(qp)
        rng = np.random.default_rng(seed)
        y = rng.standard_normal(dq.ny)
        pi = rng.standard_normal(dq.neq)
        nc = dq.C.shape[0]
        lam = rng.uniform(0.1, 2.0, nc)
        t = rng.uniform(0.1, 2.0, nc)
        smu = 0.3
        dy, dpi, dlam, dt = O.newton_step(dq, y, pi, lam, t, sigma_mu=smu)
        # the 4x4 block system of eq. (delta), assembled and solved in one piece
        ny, ne = dq.ny, dq.neq
        n = ny + ne + 2 * nc
        K = np.zeros((n, n))
        K[:ny, :ny] = dq.H
        K[:ny, ny:ny + ne] = -dq.A.T
        K[:ny, ny + ne:ny + ne + nc] = -dq.C.T
        K[ny:ny + ne, :ny] = -dq.A
        K[ny + ne:ny + ne + nc, :ny] = -dq.C
        K[ny + ne:ny + ne + nc, ny + ne + nc:] = np.eye(nc)
        K[ny + ne + nc:, ny + ne:ny + ne + nc] = np.diag(t)
        K[ny + ne + nc:, ny + ne + nc:] = np.diag(lam)
        rg = dq.H @ y - dq.A.T @ pi - dq.C.T @ lam + dq.g
        rb = -dq.A @ y + dq.b
        rd = -dq.C @ y + t + dq.d
        rm = lam * t - smu
        sol = np.linalg.solve(K, -np.concatenate([rg, rb, rd, rm]))
        np.testing.assert_allclose(dy, sol[:ny], rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(dpi, sol[ny:ny + ne], rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(dlam, sol[ny + ne:ny + ne + nc], rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(dt, sol[ny + ne + nc:], rtol=1e-9, atol=1e-10)


# ----------------------------------------------------------------------------
# invariants at convergence
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("maker", [lambda: W.small_random_qp(0), lambda: W.small_random_qp(5),
                                   lambda: W.mass_spring_qp(0),
                                   lambda: random_lq(31, N=5, boxes=True, ng=2, tight=0.5)])
def test_kkt_invariants_and_zero_gap(maker):
    """P4: stationarity, dynamics and inequality residuals, sign of (lam, t)
    and zero duality gap at the returned point."""
    qp = maker()
    res = O.solve(qp)
    assert res.status == O.CONVERGED
    rg, rb, rd, mu, mx = O.full_residuals(qp, res.y, res.pi, res.lam, res.t)
    assert max(rg, rb, rd) <= 1e-9 and mu <= 1e-9
    assert np.all(res.lam >= 0) and np.all(res.t > 0)
    dq = res.dq
    gap = O.duality_gap(dq, res.y, res.pi, res.lam[dq.active])
    obj = O.objective(dq, res.y)
    assert abs(gap) <= 1e-8 * (1 + abs(obj))


def test_symmetry_in_x0():
    """P5: zero b, q, r and symmetric boxes make the solution odd in x0."""
    a = W.small_random_qp(2)
    b = W.small_random_qp(2)
    b.b[0] = -a.b[0]
    b.x0 = -a.x0
    ra, rb_ = O.solve(a), O.solve(b)
    assert ra.status == rb_.status == O.CONVERGED
    np.testing.assert_allclose(rb_.y, -ra.y, atol=1e-9)


def test_dense_and_sparse_solves_agree():
    """P6: the dense LDL^T and the sparse LU give the same converged point."""
    qp = W.small_random_qp(4)
    a = O.solve(qp, O.IpmArg(force_dense=True))
    b = O.solve(qp, O.IpmArg(force_dense=False))
    assert a.status == b.status == O.CONVERGED
    np.testing.assert_allclose(a.y, b.y, atol=1e-10)
    np.testing.assert_allclose(a.pi, b.pi, atol=1e-9)


def test_sparse_assembly_has_the_dense_entries():
    """Large QPs are assembled as sparse matrices: the same entries as the
    dense assembly (stage-varying sizes, S != 0, general rows, masked sides,
    soft constraints), and the same converged point through the sparse LU."""
    qps = [random_lq(77, N=5, boxes=True, ng=2, tight=0.8), W.ragged_random_qp(16),
           W.soften(W.small_random_qp(2, x0_scale=2.0), range(0, 10), "u", Z=0.5, z=1.0, ls=-0.05)]
    for qp in qps:
        d, s = O.assemble(qp, sparse=False), O.assemble(qp, sparse=True)
        for name in ("H", "A", "C"):
            assert np.array_equal(getattr(d, name), getattr(s, name).toarray()), name
        for name in ("g", "b", "d", "active"):
            assert np.array_equal(getattr(d, name), getattr(s, name)), name
        a = O.solve(qp, O.IpmArg(force_dense=False), dq=d)
        b = O.solve(qp, dq=s)
        assert a.status == b.status == O.CONVERGED
        np.testing.assert_allclose(b.y, a.y, atol=1e-10)
        assert abs(O.duality_gap(s, b.y, b.pi, b.lam[s.active])) <= 1e-7


def test_equal_bound_initial_state_variant():
    """x_0 kept as a variable fixed by lb = ub box bounds (the paper's
    formulation, Sec. 2.2) gives the same solution as eliminating x_0."""
    qp = W.small_random_qp(1)
    A = qp.A[1]
    x0 = qp.x0
    qv = W.small_random_qp(1)
    qv.nx = list(qp.nx)
    qv.nx[0] = 4
    qv.A = list(qp.A)
    qv.A[0] = A
    qv.b = list(qp.b)
    qv.b[0] = np.zeros(4)
    qv.Q = list(qp.Q)
    qv.Q[0] = np.eye(4)
    qv.S = list(qp.S)
    qv.S[0] = np.zeros((2, 4))
    qv.q = list(qp.q)
    qv.q[0] = np.zeros(4)
    qv.idxbx = list(qp.idxbx)
    qv.idxbx[0] = np.arange(4)
    qv.lbx = list(qp.lbx)
    qv.lbx[0] = x0.copy()
    qv.ubx = list(qp.ubx)
    qv.ubx[0] = x0.copy()
    qv.C = list(qp.C)
    qv.C[0] = np.zeros((0, 4))
    qv.validate()
    a = O.solve(qp)
    b = O.solve(qv, O.IpmArg(tol_comp=1e-9, tol_stat=1e-9, tol_eq=1e-9, tol_ineq=1e-9))
    assert a.status == O.CONVERGED and b.status == O.CONVERGED
    sa = O.split_stages(qp, a.dq, a.y)
    sb = O.split_stages(qv, b.dq, b.y)
    np.testing.assert_allclose(sb[0][1], x0, atol=1e-7)
    for n in range(qp.N + 1):
        np.testing.assert_allclose(sb[n][0], sa[n][0], atol=1e-6)
        if n:
            np.testing.assert_allclose(sb[n][1], sa[n][1], atol=1e-6)


def test_mass_spring_batch_converges():
    """The mass-spring workload is well posed: a few instances converge."""
    for i in range(3):
        res = O.solve(W.mass_spring_qp(i))
        assert res.status == O.CONVERGED, (i, res.res)


def indefinite_lq(seed, N=8, nx=4, nu=2):
    """An OCP QP with an indefinite state cost (one negative eigenvalue of Q)
    whose reduced Hessians R + B'PB stay positive definite, x_0 eliminated,
    box bounds far outside the solution (inactive)."""
    from paper_2003_02547_gb300 import workloads as W
    rng = np.random.default_rng([77, seed])
    G = rng.standard_normal((nx, nx))
    A = G * (0.9 / max(abs(np.linalg.eigvals(G))))
    B = rng.standard_normal((nx, nu))
    b = 0.1 * rng.standard_normal(nx)
    Q = np.diag(np.r_[np.ones(nx - 1), -0.3])
    R = 3.0 * np.eye(nu)
    S = np.zeros((nu, nx))
    q = 0.5 * rng.standard_normal(nx)
    r = 0.5 * rng.standard_normal(nu)
    x0 = rng.uniform(-1, 1, nx)
    qp = W._assemble(N, A, B, b, Q, R, S, q, r, x0, 1e3, 1e3, name=f"indef{seed}")
    qp.validate()
    return qp


def reduced_hessian_min_eig(qp):
    """Smallest eigenvalue of R_n + B_n' P_{n+1} B_n over the stages of the
    classical Riccati recursion (positive: the QP is strictly convex on the
    dynamics)."""
    P = qp.Q[qp.N].copy()
    mn = np.inf
    for n in range(qp.N - 1, -1, -1):
        An, Bn = qp.A[n], qp.B[n]
        Rb = qp.R[n] + Bn.T @ P @ Bn
        Sb = qp.S[n] + Bn.T @ P @ An
        Qb = qp.Q[n] + An.T @ P @ An
        mn = min(mn, float(np.min(np.linalg.eigvalsh(Rb))))
        P = Qb - Sb.T @ np.linalg.solve(Rb, Sb)
    return mn


def test_indefinite_state_cost_matches_riccati_dp():
    """NEXT-1 pin: with Q indefinite but every reduced Hessian positive
    definite, the oracle (pivoted LDL' of the full KKT system) reaches the
    solution of the classical Riccati recursion; the stage Hessian of the last
    stage alone is indefinite, so no square-root factorisation exists."""
    for seed in range(3):
        qp = indefinite_lq(seed)
        assert reduced_hessian_min_eig(qp) > 0.1
        assert np.min(np.linalg.eigvalsh(qp.Q[qp.N])) < 0
        res = O.solve(qp)
        assert res.status == O.CONVERGED
        us, xs, pis = riccati_dp(qp)
        st = O.split_stages(qp, res.dq, res.y)
        for n in range(qp.N + 1):
            np.testing.assert_allclose(st[n][0], us[n], rtol=1e-8, atol=1e-8)
            np.testing.assert_allclose(st[n][1], xs[n], rtol=1e-8, atol=1e-8)
