"""CPU FP64 oracle for the OCP-QP primal-dual interior-point method.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
module: only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA solver.

What it computes, and the passages it follows (HPIPM paper, arXiv 2003.02547):

* ``assemble``      -- the OCP QP of Sec. 2.2 written out as the generic QP of
                       Sec. 3.1, eq. (qp):  min 1/2 y'Hy + g'y  s.t.  Ay = b,
                       Cy >= d.  Stage variables are y_n = [u_n; x_n; s^l_n;
                       s^u_n]: the slacks of the soft constraints (Sec. 2.2)
                       are ordinary primal variables here, with their
                       diagonal costs in H and g, a +1 entry in the side rows
                       they relax, and sides of their own for s >= lower
                       bound.  (The CUDA path eliminates them instead.)
* ``residuals``     -- the residual function of eq. (delta) (r_g, r_b, r_d, r_m)
                       with the Lagrangian sign convention of Sec. 3.1.
* ``newton_step``   -- eq. (delta) solved by eliminating dt then dlam (Sec. 3.3)
                       and solving the reduced KKT system eq. (kkt) with a dense
                       symmetric-indefinite LDL^T (LAPACK ?sytrf/?sytrs), or a
                       sparse LU for large systems.  No Riccati recursion.
* ``solve``         -- the infeasible-start Mehrotra predictor-corrector of
                       Sec. 4.2 in the delta formulation (Sec. 3.2, mode
                       'speed'), with the conditional corrector, the lower
                       clamp on lambda and t, and warm start (Sec. 4.2).

Conventions (fixed here, shared by the CUDA path through the C header, not
through code):

* Equality rows: for n = 0..N-1, -B_n u_n - A_n x_n + x_{n+1} = b_n, so that
  r_b = -A y + b = A_n x_n + B_n u_n + b_n - x_{n+1} and the multiplier
  pi_{n+1} of that block is the gradient of the cost-to-go at x_{n+1}.
* Inequalities: every two-sided constraint lo <= c(y) <= hi gives a lower
  side c(y) - lo >= 0 and an upper side hi - c(y) >= 0.  Per stage the
  constraint list is [box on u (idxbu order); box on x (idxbx order);
  general rows D u + C x], nc_n entries, and lambda/t hold the nc_n lower
  sides followed by the nc_n upper sides.  A side with an infinite bound is
  masked: it is left out of the arithmetic and reported as lambda = 0, t = 1.
* Soft constraints (Sec. 2.2): slack k of stage n relaxes constraint
  idxs_n[k]: its lower side becomes c(y) + s^l_k - lo >= 0 and its upper
  side hi - c(y) + s^u_k >= 0.  After the 2 nc_n constraint sides come ns_n
  sides s^l_k - lls_k >= 0 and then ns_n sides s^u_k - lus_k >= 0.

Readings where the paper is silent (the same in the CUDA path):

* start: y = 0, pi = 0, lambda = 1, t = max(1, c(y) - bound) per side;
* centring sigma = (mu_aff / mu)^3 (Mehrotra's heuristic);
* conditional corrector: keep it if mu after its step <= corr_k * mu_aff,
  otherwise take the predictor-centring direction (r_m = lambda t - sigma mu);
* step alpha = min(1, tau_b * alpha_max), tau_b = 0.995; the predictor
  uses alpha_aff = min(1, alpha_max);
* after each step lambda >= lam_min and t >= t_min (1e-16 by default);
* exit when ||r_g||inf <= tol_stat, ||r_b||inf <= tol_eq, ||r_d||inf <= tol_ineq
  and mu <= tol_comp (unscaled infinity norms), or at iter_max, or when the
  step falls below alpha_min.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

CONVERGED, MAX_ITER, MIN_STEP, NAN_FOUND = 0, 1, 2, 3

DENSE_MAX = 1500   # reduced-KKT dimension up to which the dense LDL^T is used


@dataclass
class IpmArg:
    iter_max: int = 100
    tol_stat: float = 1e-10
    tol_eq: float = 1e-10
    tol_ineq: float = 1e-10
    tol_comp: float = 1e-10
    alpha_min: float = 1e-12
    lam_min: float = 1e-16
    t_min: float = 1e-16
    tau_b: float = 0.995
    corr_k: float = 2.0
    cond_corr: bool = True
    warm_start: int = 0        # 0 none, 1 primal (y, pi), 2 primal + dual
    warm_min: float = 1e-2     # lower clamp for warm-started lambda and t
    force_dense: Optional[bool] = None


@dataclass
class DenseQp:
    """Generic-QP form of one OCP QP (Sec. 3.1, eq. qp)."""
    H: np.ndarray
    g: np.ndarray
    A: np.ndarray
    b: np.ndarray
    C: np.ndarray          # active sides only
    d: np.ndarray
    active: np.ndarray     # bool mask over the full side layout
    ny: int
    neq: int
    nside: int             # full side count, masked sides included
    var_off: list = field(default_factory=list)
    eq_off: list = field(default_factory=list)
    side_off: list = field(default_factory=list)


def _ns(qp, n: int) -> int:
    idxs = getattr(qp, "idxs", None)
    return 0 if idxs is None else len(idxs[n])


SPARSE_MIN = 5e7   # ny * (ny + sides) above which the matrices are assembled sparse


class _DenseBuilder:
    def __init__(self, shape):
        self.a = np.zeros(shape)

    def put(self, r0, c0, blk):
        blk = np.asarray(blk, dtype=np.float64)
        self.a[r0:r0 + blk.shape[0], c0:c0 + blk.shape[1]] = blk

    def row(self, r, cols, vals):
        self.a[r, cols] = vals

    def done(self):
        return self.a


class _SparseBuilder:
    """The same entries as _DenseBuilder, kept as triplets (a block's zeros
    included), for QPs whose dense matrices would not fit in memory."""

    def __init__(self, shape):
        self.shape = shape
        self.r, self.c, self.v = [], [], []

    def put(self, r0, c0, blk):
        blk = np.asarray(blk, dtype=np.float64)
        h, w = blk.shape
        rr, cc = np.meshgrid(np.arange(r0, r0 + h), np.arange(c0, c0 + w), indexing="ij")
        self.r.append(rr.ravel())
        self.c.append(cc.ravel())
        self.v.append(blk.ravel())

    def row(self, r, cols, vals):
        cols = np.atleast_1d(np.asarray(cols))
        self.r.append(np.full(cols.size, r))
        self.c.append(cols)
        self.v.append(np.atleast_1d(np.asarray(vals, dtype=np.float64)))

    def done(self):
        if not self.r:
            return scipy.sparse.csr_matrix(self.shape)
        r, c, v = np.concatenate(self.r), np.concatenate(self.c), np.concatenate(self.v)
        # later entries overwrite earlier ones at the same position (as in the dense builder)
        key = r.astype(np.int64) * self.shape[1] + c
        _, last = np.unique(key[::-1], return_index=True)
        keep = key.size - 1 - last
        return scipy.sparse.csr_matrix((v[keep], (r[keep], c[keep])), shape=self.shape)


def assemble(qp, sparse: Optional[bool] = None) -> DenseQp:
    """Write the stage-wise OCP QP (Sec. 2.2) as one generic QP; H, A and C
    are dense arrays, or scipy.sparse CSR matrices with the same entries for
    QPs too large for dense storage (``sparse=None`` decides by size)."""
    N = qp.N
    ns = [_ns(qp, n) for n in range(N + 1)]
    nv = [qp.nx[n] + qp.nu[n] + 2 * ns[n] for n in range(N + 1)]
    var_off = np.concatenate([[0], np.cumsum(nv)]).astype(int)
    ny = int(var_off[-1])
    eq_sz = [qp.nx[n + 1] for n in range(N)]
    eq_off = np.concatenate([[0], np.cumsum(eq_sz)]).astype(int)
    neq = int(eq_off[-1])
    nc = [qp.nbu(n) + qp.nbx(n) + qp.ng(n) for n in range(N + 1)]
    side_off = np.concatenate([[0], np.cumsum([2 * nc[n] + 2 * ns[n] for n in range(N + 1)])]).astype(int)
    nside = int(side_off[-1])
    if sparse is None:
        sparse = float(ny) * float(ny + nside) > SPARSE_MIN
    Builder = _SparseBuilder if sparse else _DenseBuilder

    Hb = Builder((ny, ny))
    g = np.zeros(ny)
    for n in range(N + 1):
        o, nu, nx = var_off[n], qp.nu[n], qp.nx[n]
        Hb.put(o, o, qp.R[n])
        Hb.put(o, o + nu, qp.S[n])
        Hb.put(o + nu, o, qp.S[n].T)
        Hb.put(o + nu, o + nu, qp.Q[n])
        g[o:o + nu] = qp.r[n]
        g[o + nu:o + nu + nx] = qp.q[n]
        for k in range(ns[n]):
            # slack costs 1/2 Z s^2 + z s, s^l block then s^u block
            jl, ju = o + nu + nx + k, o + nu + nx + ns[n] + k
            Hb.row(jl, jl, qp.Zl[n][k])
            Hb.row(ju, ju, qp.Zu[n][k])
            g[jl] = qp.zl[n][k]
            g[ju] = qp.zu[n][k]
    H = Hb.done()

    Ab = Builder((neq, ny))
    b = np.zeros(neq)
    for n in range(N):
        r0 = eq_off[n]
        o, nu, nx = var_off[n], qp.nu[n], qp.nx[n]
        Ab.put(r0, o, -qp.B[n])
        Ab.put(r0, o + nu, -qp.A[n])
        o1, nu1, nx1 = var_off[n + 1], qp.nu[n + 1], qp.nx[n + 1]
        Ab.put(r0, o1 + nu1, np.eye(nx1))
        b[eq_off[n]:eq_off[n + 1]] = qp.b[n]
    A = Ab.done()

    Cb = Builder((nside, ny))
    dfull = np.zeros(nside)
    active = np.zeros(nside, dtype=bool)
    for n in range(N + 1):
        o, nu = var_off[n], qp.nu[n]
        rows = []   # (columns, values) of each constraint row c(y)
        lo = []
        hi = []
        for k, i in enumerate(qp.idxbu[n]):
            rows.append((np.array([o + int(i)]), np.array([1.0])))
            lo.append(qp.lbu[n][k])
            hi.append(qp.ubu[n][k])
        for k, i in enumerate(qp.idxbx[n]):
            rows.append((np.array([o + nu + int(i)]), np.array([1.0])))
            lo.append(qp.lbx[n][k])
            hi.append(qp.ubx[n][k])
        cols_g = np.arange(o, o + nu + qp.nx[n])
        for k in range(qp.ng(n)):
            rows.append((cols_g, np.concatenate([qp.D[n][k], qp.C[n][k]])))
            lo.append(qp.lg[n][k])
            hi.append(qp.ug[n][k])
        c = len(rows)
        s = side_off[n]
        for k in range(c):
            # lower side: c(y) - lo >= 0 ; upper side: -c(y) + hi >= 0
            cols, vals = rows[k]
            Cb.row(s + k, cols, vals)
            dfull[s + k] = lo[k]
            active[s + k] = np.isfinite(lo[k])
            Cb.row(s + c + k, cols, -vals)
            dfull[s + c + k] = -hi[k]
            active[s + c + k] = np.isfinite(hi[k])
        m = ns[n]
        for k in range(m):
            # slack k relaxes both sides of constraint idxs[k] and has a
            # lower bound of its own on each
            ci = int(qp.idxs[n][k])
            jl, ju = o + nu + qp.nx[n] + k, o + nu + qp.nx[n] + m + k
            Cb.row(s + ci, jl, 1.0)
            Cb.row(s + c + ci, ju, 1.0)
            Cb.row(s + 2 * c + k, jl, 1.0)
            dfull[s + 2 * c + k] = qp.lls[n][k]
            active[s + 2 * c + k] = True
            Cb.row(s + 2 * c + m + k, ju, 1.0)
            dfull[s + 2 * c + m + k] = qp.lus[n][k]
            active[s + 2 * c + m + k] = True
    Crow = Cb.done()
    C = Crow[np.flatnonzero(active)] if sparse else Crow[active]
    return DenseQp(H=H, g=g, A=A, b=b, C=C, d=dfull[active], active=active,
                   ny=ny, neq=neq, nside=nside, var_off=list(var_off),
                   eq_off=list(eq_off), side_off=list(side_off))


def residuals(dq: DenseQp, y, pi, lam, t):
    """Residual function of eq. (delta): r_g, r_b, r_d (active sides) and
    the duality measure mu = lam't / n_c."""
    rg = dq.H @ y + dq.g - dq.A.T @ pi - dq.C.T @ lam
    rb = -dq.A @ y + dq.b
    rd = -dq.C @ y + dq.d + t
    nc = lam.size
    mu = float(lam @ t) / nc if nc else 0.0
    return rg, rb, rd, mu


class KktFactor:
    """Factorisation of the reduced KKT matrix of eq. (kkt) at fixed (lam, t)."""

    def __init__(self, dq: DenseQp, lam, t, force_dense: Optional[bool] = None):
        self.dq = dq
        self.lam = lam
        self.t = t
        W = lam / t
        n = dq.ny + dq.neq
        self.n = n
        if scipy.sparse.issparse(dq.H):
            # sparse assembly (large QPs): the same Ht with sparse products
            Ht = dq.H + dq.C.T @ scipy.sparse.diags(W) @ dq.C
            dense = False
        else:
            Ht = dq.H + dq.C.T @ (W[:, None] * dq.C)
            dense = (n <= DENSE_MAX) if force_dense is None else force_dense
        self.dense = dense
        if dense:
            K = np.zeros((n, n))
            K[:dq.ny, :dq.ny] = Ht
            K[:dq.ny, dq.ny:] = -dq.A.T
            K[dq.ny:, :dq.ny] = -dq.A
            # symmetric-indefinite LDL^T (Bunch-Kaufman), LAPACK dsytrf
            lu, ipiv, info = scipy.linalg.lapack.dsytrf(K, lower=1)
            if info != 0:
                raise np.linalg.LinAlgError(f"dsytrf info={info}")
            self.lu, self.ipiv = lu, ipiv
        else:
            Ks = scipy.sparse.bmat([[scipy.sparse.csc_matrix(Ht), scipy.sparse.csc_matrix(-dq.A.T)],
                                    [scipy.sparse.csc_matrix(-dq.A), None]], format="csc")
            self.splu = scipy.sparse.linalg.splu(Ks)

    def solve_reduced(self, rhs):
        if self.dense:
            x, info = scipy.linalg.lapack.dsytrs(self.lu, self.ipiv, rhs, lower=1)
            if info != 0:
                raise np.linalg.LinAlgError(f"dsytrs info={info}")
            return x
        return self.splu.solve(rhs)

    def step(self, rg, rb, rd, rm):
        """Newton step of eq. (delta): eliminate dt = C dy - r_d and
        dlam = -T^{-1}(r_m + Lam dt) (Sec. 3.3), solve eq. (kkt) for (dy, dpi)."""
        dq, lam, t = self.dq, self.lam, self.t
        W = lam / t
        gt = rg - dq.C.T @ (W * rd - rm / t)
        rhs = -np.concatenate([gt, rb])
        sol = self.solve_reduced(rhs)
        dy = sol[:dq.ny]
        dpi = sol[dq.ny:]
        dt = dq.C @ dy - rd
        dlam = -(rm + lam * dt) / t
        return dy, dpi, dlam, dt


def newton_step(dq: DenseQp, y, pi, lam, t, sigma_mu: float = 0.0, force_dense=None):
    """One Newton direction of eq. (delta) at the given iterate with
    r_m = lam*t - sigma_mu (sigma_mu = 0: affine predictor)."""
    rg, rb, rd, _ = residuals(dq, y, pi, lam, t)
    rm = lam * t - sigma_mu
    return KktFactor(dq, lam, t, force_dense).step(rg, rb, rd, rm)


def _max_step(lam, t, dlam, dt) -> float:
    """Largest alpha >= 0 with lam + alpha dlam >= 0 and t + alpha dt >= 0
    (inf when no component decreases)."""
    a = np.inf
    neg = dlam < 0
    if np.any(neg):
        a = min(a, float(np.min(-lam[neg] / dlam[neg])))
    neg = dt < 0
    if np.any(neg):
        a = min(a, float(np.min(-t[neg] / dt[neg])))
    return a


@dataclass
class IpmResult:
    y: np.ndarray
    pi: np.ndarray
    lam: np.ndarray        # full side layout (masked sides 0)
    t: np.ndarray          # full side layout (masked sides 1)
    status: int
    iters: int
    res: tuple             # (||r_g||inf, ||r_b||inf, ||r_d||inf, mu) at exit
    history: list = field(default_factory=list)
    dq: Optional[DenseQp] = None


def initial_point(dq: DenseQp, y=None, pi=None, lam=None, t=None, arg: IpmArg = IpmArg()):
    """Start point (reading: y = 0, pi = 0, lam = 1, t = max(1, Cy - d));
    warm start 1 keeps the given (y, pi), warm start 2 also the given
    (lam, t) clamped below by warm_min (Sec. 4.2: warm start of the primal,
    or of the primal and dual variables)."""
    if arg.warm_start >= 1 and y is not None:
        y = np.array(y, dtype=np.float64)
        pi = np.zeros(dq.neq) if pi is None else np.array(pi, dtype=np.float64)
    else:
        y = np.zeros(dq.ny)
        pi = np.zeros(dq.neq)
    if arg.warm_start >= 2 and lam is not None and t is not None:
        lam = np.maximum(np.asarray(lam, dtype=np.float64)[dq.active], arg.warm_min)
        t = np.maximum(np.asarray(t, dtype=np.float64)[dq.active], arg.warm_min)
    else:
        lam = np.ones(dq.C.shape[0])
        t = np.maximum(1.0, dq.C @ y - dq.d)
    return y, pi, lam, t


def expand_sides(dq: DenseQp, v, fill):
    out = np.full(dq.nside, fill, dtype=np.float64)
    out[dq.active] = v
    return out


def solve(qp, arg: IpmArg = IpmArg(), y0=None, pi0=None, lam0=None, t0=None,
          dq: Optional[DenseQp] = None, record: bool = False) -> IpmResult:
    """Infeasible-start Mehrotra predictor-corrector IPM (Sec. 4.2) in the
    delta formulation (Sec. 3.2), residual-based exit (mode 'speed')."""
    if dq is None:
        dq = assemble(qp)
    y, pi, lam, t = initial_point(dq, y0, pi0, lam0, t0, arg)
    nc = lam.size
    status = MAX_ITER
    it = 0
    alpha = 1.0
    hist = []
    while True:
        rg, rb, rd, mu = residuals(dq, y, pi, lam, t)
        res = (np.max(np.abs(rg), initial=0.0), np.max(np.abs(rb), initial=0.0),
               np.max(np.abs(rd), initial=0.0), mu)
        if record:
            hist.append(dict(y=y.copy(), pi=pi.copy(), lam=lam.copy(), t=t.copy(), res=res, alpha=alpha))
        if not all(np.isfinite(res)):
            status = NAN_FOUND
            break
        if (res[0] <= arg.tol_stat and res[1] <= arg.tol_eq and res[2] <= arg.tol_ineq
                and res[3] <= arg.tol_comp):
            status = CONVERGED
            break
        if it >= arg.iter_max:
            status = MAX_ITER
            break
        if it > 0 and alpha < arg.alpha_min:
            status = MIN_STEP
            break
        fac = KktFactor(dq, lam, t, arg.force_dense)
        # predictor (affine) direction: r_m = lam * t
        rm = lam * t
        dy, dpi, dlam, dt = fac.step(rg, rb, rd, rm)
        if nc:
            a_aff = min(1.0, _max_step(lam, t, dlam, dt))
            mu_aff = float((lam + a_aff * dlam) @ (t + a_aff * dt)) / nc
            sigma = (mu_aff / mu) ** 3 if mu > 0 else 0.0
            # Mehrotra corrector: second-order term and centring
            rm_c = lam * t + dlam * dt - sigma * mu
            cdy, cdpi, cdlam, cdt = fac.step(rg, rb, rd, rm_c)
            use_corr = True
            if arg.cond_corr:
                a_c = min(1.0, _max_step(lam, t, cdlam, cdt))
                mu_c = float((lam + a_c * cdlam) @ (t + a_c * cdt)) / nc
                use_corr = mu_c <= arg.corr_k * mu_aff
            if use_corr:
                dy, dpi, dlam, dt = cdy, cdpi, cdlam, cdt
            else:
                rm_pc = lam * t - sigma * mu
                dy, dpi, dlam, dt = fac.step(rg, rb, rd, rm_pc)
            alpha = min(1.0, arg.tau_b * _max_step(lam, t, dlam, dt))
        else:
            alpha = 1.0
        y = y + alpha * dy
        pi = pi + alpha * dpi
        lam = np.maximum(lam + alpha * dlam, arg.lam_min)
        t = np.maximum(t + alpha * dt, arg.t_min)
        it += 1
    return IpmResult(y=y, pi=pi, lam=expand_sides(dq, lam, 0.0), t=expand_sides(dq, t, 1.0),
                     status=status, iters=it, res=res, history=hist, dq=dq)


def full_residuals(qp, y, pi, lam_full, t_full, dq: Optional[DenseQp] = None):
    """KKT residual norms of a candidate solution given in the full side
    layout: (||r_g||inf, ||r_b||inf, ||r_d||inf, mu, max_i lam_i t_i)."""
    if dq is None:
        dq = assemble(qp)
    lam = np.asarray(lam_full)[dq.active]
    t = np.asarray(t_full)[dq.active]
    rg, rb, rd, mu = residuals(dq, np.asarray(y), np.asarray(pi), lam, t)
    mx = float(np.max(lam * t)) if lam.size else 0.0
    return (float(np.max(np.abs(rg), initial=0.0)), float(np.max(np.abs(rb), initial=0.0)),
            float(np.max(np.abs(rd), initial=0.0)), mu, mx)


def objective(dq: DenseQp, y) -> float:
    return 0.5 * float(y @ dq.H @ y) + float(dq.g @ y)


def duality_gap(dq: DenseQp, y, pi, lam_act) -> float:
    """Primal objective minus the Lagrangian dual objective
    -1/2 y'Hy + b'pi + d'lam (valid where Hy + g - A'pi - C'lam = 0)."""
    dual = -0.5 * float(y @ dq.H @ y) + float(dq.b @ pi) + float(dq.d @ lam_act)
    return objective(dq, y) - dual


def split_slacks(qp, dq: DenseQp, y):
    """y -> list of (s^l_n, s^u_n)."""
    out = []
    for n in range(qp.N + 1):
        o = dq.var_off[n] + qp.nu[n] + qp.nx[n]
        m = _ns(qp, n)
        out.append((y[o:o + m], y[o + m:o + 2 * m]))
    return out


def split_stages(qp, dq: DenseQp, y):
    """y -> list of (u_n, x_n)."""
    out = []
    for n in range(qp.N + 1):
        o = dq.var_off[n]
        nu, nx = qp.nu[n], qp.nx[n]
        out.append((y[o:o + nu], y[o + nu:o + nu + nx]))
    return out
