"""Seeded synthetic OCP-QP instances shaped like the paper's workloads.

This module builds problem data only.  It holds none of the interior-point
method's arithmetic and imports neither the solver nor the oracle, so both the
CUDA path and the CPU oracle can take their inputs from here.

Problem statement (Sec. 2.2, the OCP QP): for stages n = 0..N the variables are
y_n = [u_n; x_n] (controls first), the cost is
    1/2 [u;x;1]^T [[R, S, r], [S^T, Q, q], [r^T, q^T, 0]] [u;x;1]
with S_n of shape (nu_n, nx_n), the dynamics are
    x_{n+1} = A_n x_n + B_n u_n + b_n,       n = 0..N-1,
and the inequalities are two-sided boxes on selected components of u_n and
x_n plus general constraints lg_n <= D_n u_n + C_n x_n <= ug_n.  A side whose
bound is +-inf is masked out (Sec. 2.1: single sides can be deactivated).

The initial state is handled by elimination: the workloads fix x_0 = x0, so
stage 0 carries no state (nx_0 = 0) and x0 enters the data of stage 0 as
b_0 = A x0 + b, r_0 = r + S x0 and lg_0/ug_0 shifted by -C x0.  Stage-wise
sizes are allowed to vary (Sec. 2.2), so this is the same QP in the remaining
variables; the paper's alternative (x_0 boxed with equal bounds) is also
expressible with this container and is used by a test.

Every generator is deterministic in its seed: ``numpy.random.default_rng``
is seeded with ``[config_id, qp_index, redraw]``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

INF = np.inf


@dataclass
class OcpQp:
    """One OCP QP in stage-wise form (Sec. 2.2).  Lists are indexed by stage.

    Shapes: A[n] (nx[n+1], nx[n]); B[n] (nx[n+1], nu[n]); b[n] (nx[n+1],)
    for n < N.  Q[n] (nx[n], nx[n]); S[n] (nu[n], nx[n]); R[n] (nu[n], nu[n]);
    q[n] (nx[n],); r[n] (nu[n],) for n <= N.  idxbu[n]/idxbx[n] are int
    index lists into u_n / x_n with bounds lbu/ubu and lbx/ubx; C[n] (ng, nx[n]),
    D[n] (ng, nu[n]) with bounds lg/ug.  Objects may be shared between stages
    and between QPs (time-invariant data); ``stage_key[n]`` names the data
    block stage n uses, equal keys meaning bit-identical data.
    """

    N: int
    nx: List[int]
    nu: List[int]
    A: List[np.ndarray]
    B: List[np.ndarray]
    b: List[np.ndarray]
    Q: List[np.ndarray]
    S: List[np.ndarray]
    R: List[np.ndarray]
    q: List[np.ndarray]
    r: List[np.ndarray]
    idxbu: List[np.ndarray]
    lbu: List[np.ndarray]
    ubu: List[np.ndarray]
    idxbx: List[np.ndarray]
    lbx: List[np.ndarray]
    ubx: List[np.ndarray]
    C: List[np.ndarray]
    D: List[np.ndarray]
    lg: List[np.ndarray]
    ug: List[np.ndarray]
    x0: Optional[np.ndarray] = None
    stage_key: List[object] = field(default_factory=list)
    name: str = ""
    # soft constraints (Sec. 2.2): idxs[n] (ns_n,) indexes the stage's
    # constraint list [box u; box x; general]; slack k relaxes the lower side
    # of constraint idxs[n][k] by s^l_k and its upper side by s^u_k, with
    # cost 1/2 Zl s^l^2 + zl s^l (Zu, zu for s^u) and s^l >= lls, s^u >= lus.
    # None: no slacks.
    idxs: Optional[List[np.ndarray]] = None
    Zl: Optional[List[np.ndarray]] = None
    Zu: Optional[List[np.ndarray]] = None
    zl: Optional[List[np.ndarray]] = None
    zu: Optional[List[np.ndarray]] = None
    lls: Optional[List[np.ndarray]] = None
    lus: Optional[List[np.ndarray]] = None

    def ng(self, n: int) -> int:
        return self.C[n].shape[0]

    def ns(self, n: int) -> int:
        return 0 if self.idxs is None else len(self.idxs[n])

    def nbu(self, n: int) -> int:
        return len(self.idxbu[n])

    def nbx(self, n: int) -> int:
        return len(self.idxbx[n])

    def dims(self):
        """Per-stage (nx, nu, nbx, nbu, ng) tuples, n = 0..N."""
        return [(self.nx[n], self.nu[n], self.nbx(n), self.nbu(n), self.ng(n))
                for n in range(self.N + 1)]

    def validate(self) -> None:
        N = self.N
        assert len(self.nx) == N + 1 and len(self.nu) == N + 1
        for n in range(N):
            assert self.A[n].shape == (self.nx[n + 1], self.nx[n])
            assert self.B[n].shape == (self.nx[n + 1], self.nu[n])
            assert self.b[n].shape == (self.nx[n + 1],)
        for n in range(N + 1):
            nx, nu = self.nx[n], self.nu[n]
            assert self.Q[n].shape == (nx, nx)
            assert self.S[n].shape == (nu, nx)
            assert self.R[n].shape == (nu, nu)
            assert self.q[n].shape == (nx,) and self.r[n].shape == (nu,)
            ng = self.C[n].shape[0]
            assert self.C[n].shape == (ng, nx) and self.D[n].shape == (ng, nu)
            assert self.lg[n].shape == (ng,) and self.ug[n].shape == (ng,)
            assert len(self.lbu[n]) == len(self.idxbu[n]) == len(self.ubu[n])
            assert len(self.lbx[n]) == len(self.idxbx[n]) == len(self.ubx[n])
            if len(self.idxbu[n]):
                assert 0 <= min(self.idxbu[n]) and max(self.idxbu[n]) < nu
            if len(self.idxbx[n]):
                assert 0 <= min(self.idxbx[n]) and max(self.idxbx[n]) < nx
            ns = self.ns(n)
            if ns:
                nc = self.nbu(n) + self.nbx(n) + ng
                idx = np.asarray(self.idxs[n])
                assert 0 <= idx.min() and idx.max() < nc and len(set(idx.tolist())) == ns
                for arr in (self.Zl, self.Zu, self.zl, self.zu, self.lls, self.lus):
                    assert np.asarray(arr[n]).shape == (ns,)
                assert np.all(np.asarray(self.Zl[n]) >= 0) and np.all(np.asarray(self.Zu[n]) >= 0)
                assert np.all(np.isfinite(self.lls[n])) and np.all(np.isfinite(self.lus[n]))


def _rng(cfg: int, index: int, redraw: int = 0) -> np.random.Generator:
    return np.random.default_rng([cfg, index, redraw])


def _stable_A(rng: np.random.Generator, nx: int, radius: float = 0.95) -> np.ndarray:
    """Gaussian matrix rescaled to the given spectral radius."""
    G = rng.standard_normal((nx, nx))
    rho = np.max(np.abs(np.linalg.eigvals(G)))
    return G * (radius / rho)


def _assemble(N, A, B, b, Q, R, S, q, r, x0, ubound, xbound, ng=0, C=None, D=None,
              lg=None, ug=None, name="", shared_key=None) -> OcpQp:
    """Time-invariant OCP QP with x_0 = x0 eliminated (nx_0 = 0).

    Stage-0 data is built from x0; stages 1..N-1 share one data block and
    stage N (terminal, no control) another.
    """
    nx = A.shape[0]
    nu = B.shape[1]
    Z = np.zeros
    nxs = [0] + [nx] * N
    nus = [nu] * N + [0]
    A_l, B_l, b_l = [], [], []
    Q_l, S_l, R_l, q_l, r_l = [], [], [], [], []
    ibu, lbu, ubu, ibx, lbx, ubx = [], [], [], [], [], []
    C_l, D_l, lg_l, ug_l = [], [], [], []
    for n in range(N + 1):
        if n < N:
            if n == 0:
                A_l.append(Z((nx, 0)))
                b_l.append(A @ x0 + b)
            else:
                A_l.append(A)
                b_l.append(b)
            B_l.append(B)
        nxn, nun = nxs[n], nus[n]
        Q_l.append(Q if nxn else Z((0, 0)))
        R_l.append(R if nun else Z((0, 0)))
        if n == 0:
            S_l.append(Z((nu, 0)))
            q_l.append(Z(0))
            r_l.append(r + S @ x0)
        else:
            S_l.append(S if nun else Z((0, nx)))
            q_l.append(q)
            r_l.append(r if nun else Z(0))
        ibu.append(np.arange(nun, dtype=np.int64))
        lbu.append(-ubound * np.ones(nun))
        ubu.append(ubound * np.ones(nun))
        ibx.append(np.arange(nxn, dtype=np.int64))
        lbx.append(-xbound * np.ones(nxn))
        ubx.append(xbound * np.ones(nxn))
        if ng:
            Cn, Dn, lgn, ugn = C[n], D[n], lg[n], ug[n]
            if n == 0:
                ugn = ugn - Cn @ x0
                lgn = lgn - Cn @ x0
                Cn = Z((ng, 0))
            if not nun:
                Dn = Z((ng, 0))
            C_l.append(Cn)
            D_l.append(Dn)
            lg_l.append(lgn)
            ug_l.append(ugn)
        else:
            C_l.append(Z((0, nxn)))
            D_l.append(Z((0, nun)))
            lg_l.append(Z(0))
            ug_l.append(Z(0))
    key = shared_key if shared_key is not None else name
    stage_key = [(name, 0)] + [(key, "mid") if (n < N and ng == 0) else (name, n)
                               for n in range(1, N)] + [(key, "term") if ng == 0 else (name, N)]
    qp = OcpQp(N=N, nx=nxs, nu=nus, A=A_l, B=B_l, b=b_l, Q=Q_l, S=S_l, R=R_l, q=q_l, r=r_l,
               idxbu=ibu, lbu=lbu, ubu=ubu, idxbx=ibx, lbx=lbx, ubx=ubx,
               C=C_l, D=D_l, lg=lg_l, ug=ug_l, x0=np.array(x0, dtype=np.float64),
               stage_key=stage_key, name=name)
    # x0-dependent stage-0 terms, kept so that x0 can be replaced later
    qp.S_full = S
    qp.C0_full = C[0] if ng else None
    return qp


# --------------------------------------------------------------------------
# Workload 0: one small random QP (N=10, nx=4, nu=2), plain FP64 IPM.
# --------------------------------------------------------------------------
def small_random_qp(index: int = 0, N: int = 10, nx: int = 4, nu: int = 2,
                    x0_scale: float = 1.0, cfg: int = 0) -> OcpQp:
    """A with spectral radius 0.95 (Gaussian, rescaled), B ~ N(0,1), b = 0,
    Q = I, R = 0.1 I, S = 0, q = r = 0, |u| <= 1, |x| <= 5,
    x0 ~ U[-2, 2]^nx (times ``x0_scale``)."""
    rng = _rng(cfg, index)
    A = _stable_A(rng, nx)
    B = rng.standard_normal((nx, nu))
    x0 = rng.uniform(-2.0, 2.0, nx) * x0_scale
    return _assemble(N, A, B, np.zeros(nx), np.eye(nx), 0.1 * np.eye(nu), np.zeros((nu, nx)),
                     np.zeros(nx), np.zeros(nu), x0, ubound=1.0, xbound=5.0,
                     name=f"small{cfg}_{index}")


# --------------------------------------------------------------------------
# Workload 1: linear mass-spring chain (Sec. 5.1), 8 masses, N = 30.
# --------------------------------------------------------------------------
def mass_spring_model(M: int = 8, dt: float = 0.5, k: float = 1.0, m: float = 1.0,
                      scheme: str = "symplectic"):
    """Chain of M masses between two walls joined by springs of stiffness k;
    forces act on the first M-1 masses (Sec. 5.1: nx = 2M, nu = M-1).
    State x = [positions p; velocities v], continuous model
    pdot = v, vdot = (k/m) T p + F u / m with T = tridiag(1, -2, 1) and
    F = [I_{M-1}; 0].

    ``scheme="symplectic"`` (default) is the semi-implicit Euler step
    v+ = v + dt vdot(p, u), p+ = p + dt v+.  ``scheme="explicit"`` is the
    forward Euler step A = I + dt Ac, B = dt Bc, whose spectral radius is
    about 1.40 at dt = 0.5: with |u| <= 0.5 and |x| <= 4 over N = 30 stages
    those QPs have no feasible point, so the workload uses the
    semi-implicit step (spectral radius 1, like the exact discretisation).
    """
    T = -2.0 * np.eye(M) + np.eye(M, k=1) + np.eye(M, k=-1)
    F = np.eye(M, M - 1)
    K = (k / m) * T
    if scheme == "explicit":
        Ac = np.zeros((2 * M, 2 * M))
        Ac[:M, M:] = np.eye(M)
        Ac[M:, :M] = K
        Bc = np.zeros((2 * M, M - 1))
        Bc[M:, :] = F / m
        return np.eye(2 * M) + dt * Ac, dt * Bc
    if scheme != "symplectic":
        raise ValueError(scheme)
    A = np.block([[np.eye(M) + dt * dt * K, dt * np.eye(M)],
                  [dt * K, np.eye(M)]])
    B = np.vstack([dt * dt * F / m, dt * F / m])
    return A, B


def mass_spring_qp(index: int, M: int = 8, N: int = 30, cfg: int = 1,
                   x0: Optional[np.ndarray] = None) -> OcpQp:
    """Q = I, R = I, |u| <= 0.5, |x| <= 4, x0 ~ U[-1, 1]^(2M); all QPs of
    the batch share the model and differ only in x0."""
    A, B = mass_spring_model(M)
    nx, nu = A.shape[0], B.shape[1]
    if x0 is None:
        x0 = _rng(cfg, index).uniform(-1.0, 1.0, nx)
    return _assemble(N, A, B, np.zeros(nx), np.eye(nx), np.eye(nu), np.zeros((nu, nx)),
                     np.zeros(nx), np.zeros(nu), x0, ubound=0.5, xbound=4.0,
                     name=f"ms{cfg}_{index}", shared_key=f"massspring{M}_{N}")


def mass_spring_batch(count: int = 1024, M: int = 8, N: int = 30) -> List[OcpQp]:
    return [mass_spring_qp(i, M=M, N=N) for i in range(count)]


# --------------------------------------------------------------------------
# Workload 2: ragged batch of random QPs with general constraints.
# --------------------------------------------------------------------------
def ragged_random_qp(index: int, cfg: int = 2, N_range=(10, 100), nx_range=(4, 64),
                     max_redraw: int = 100) -> OcpQp:
    """N ~ U{10..100}, nx ~ U{4..64}, nu ~ U{2..floor(nx/2)}, ng = floor(nx/4)
    one-sided general constraints C x + D u <= d with C, D ~ N(0,1) at every
    stage; otherwise as the small random QP.  d_n = C_n xbar_n + s_n with
    s_n ~ U[0.1, 1] along the zero-input trajectory xbar (xbar_0 = x0,
    xbar_{n+1} = A xbar_n), so (xbar, 0) is strictly feasible; draws whose
    xbar leaves |x| < 5 are redrawn with the next ``redraw`` seed."""
    for redraw in range(max_redraw):
        rng = _rng(cfg, index, redraw)
        N = int(rng.integers(N_range[0], N_range[1] + 1))
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        nu = int(rng.integers(2, nx // 2 + 1))
        ng = nx // 4
        A = _stable_A(rng, nx)
        B = rng.standard_normal((nx, nu))
        x0 = rng.uniform(-2.0, 2.0, nx)
        xbar = [x0]
        for _ in range(N):
            xbar.append(A @ xbar[-1])
        if max(np.max(np.abs(v)) for v in xbar) >= 5.0 * 0.98:
            continue
        C = [rng.standard_normal((ng, nx)) for _ in range(N + 1)]
        D = [rng.standard_normal((ng, nu)) for _ in range(N + 1)]
        s = [rng.uniform(0.1, 1.0, ng) for _ in range(N + 1)]
        ug = [C[n] @ xbar[n] + s[n] for n in range(N + 1)]
        lg = [-INF * np.ones(ng) for _ in range(N + 1)]
        qp = _assemble(N, A, B, np.zeros(nx), np.eye(nx), 0.1 * np.eye(nu), np.zeros((nu, nx)),
                       np.zeros(nx), np.zeros(nu), x0, ubound=1.0, xbound=5.0, ng=ng,
                       C=C, D=D, lg=lg, ug=ug, name=f"rag{cfg}_{index}_{redraw}")
        qp.redraws = redraw
        return qp
    raise RuntimeError(f"no feasible draw for ragged QP {index}")


def ragged_batch(count: int = 4096, cfg: int = 2) -> List[OcpQp]:
    return [ragged_random_qp(i, cfg=cfg) for i in range(count)]


# --------------------------------------------------------------------------
# Workload 4: large-stage batch (N = 100, nx = 128, nu = 64).
# --------------------------------------------------------------------------
def large_stage_qp(index: int, cfg: int = 4, N: int = 100, nx: int = 128, nu: int = 64) -> OcpQp:
    """A as in the small random QP (spectral radius 0.95), B ~ N(0, 1/sqrt(nx))
    (standard deviation 1/sqrt(nx)), Q = I, R = 0.5 I, |x| <= 5, |u| <= 1,
    x0 ~ U[-2, 2]^nx."""
    rng = _rng(cfg, index)
    A = _stable_A(rng, nx)
    B = rng.standard_normal((nx, nu)) / np.sqrt(nx)
    x0 = rng.uniform(-2.0, 2.0, nx)
    return _assemble(N, A, B, np.zeros(nx), np.eye(nx), 0.5 * np.eye(nu), np.zeros((nu, nx)),
                     np.zeros(nx), np.zeros(nu), x0, ubound=1.0, xbound=5.0,
                     name=f"large{cfg}_{index}")


def large_stage_batch(count: int = 256, **kw) -> List[OcpQp]:
    return [large_stage_qp(i, **kw) for i in range(count)]


# --------------------------------------------------------------------------
# Workload 3: serving arrivals.
# --------------------------------------------------------------------------
@dataclass
class Arrival:
    t: float            # arrival time in seconds from the start
    key: int            # request key; a repeat reuses an earlier key
    qp: OcpQp
    warm: bool          # True for a repeat that may warm start


def serving_arrivals(rate: float = 20000.0, duration: float = 1.0, repeat_frac: float = 0.3,
                     cfg: int = 3, seed_pool: int = 4096, x0_sigma: float = 0.01) -> List[Arrival]:
    """Open-loop Poisson arrivals at ``rate`` QP/s.  A fraction ``repeat_frac``
    repeats an earlier key with x0 perturbed by N(0, x0_sigma^2) (standard
    deviation x0_sigma); the rest are fresh ragged random QPs."""
    rng = np.random.default_rng([cfg, 0, 0])
    t = 0.0
    out: List[Arrival] = []
    keys: List[int] = []
    base: dict = {}
    pool: dict = {}
    nxt = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        if keys and rng.uniform() < repeat_frac:
            key = int(keys[int(rng.integers(0, len(keys)))])
            src = base[key]
            x0 = src.x0 + x0_sigma * rng.standard_normal(src.x0.shape)
            qp = perturb_x0(src, x0)
            out.append(Arrival(t, key, qp, True))
        else:
            key = nxt
            nxt += 1
            idx = key % seed_pool
            if idx not in pool:
                pool[idx] = ragged_random_qp(idx, cfg=2)
            qp = pool[idx]
            base[key] = qp
            keys.append(key)
            out.append(Arrival(t, key, qp, False))
    return out


def soften(qp: OcpQp, stages, which: str = "x", Z: float = 1.0, z: float = 1.0, ls: float = 0.0) -> OcpQp:
    """Copy of ``qp`` whose constraints of kind ``which`` ("u": boxes on u,
    "x": boxes on x, "g": general rows, "all") at ``stages`` are soft, with
    Zl = Zu = Z, zl = zu = z and slack lower bounds ls (Sec. 2.2)."""
    import copy
    new = copy.copy(qp)
    N = qp.N
    idxs, Zl, Zu, zl, zu, lls, lus = ([np.zeros(0, dtype=np.int32) if k == 0 else np.zeros(0)
                                       for _ in range(N + 1)] for k in range(7))
    for n in stages:
        nbu, nbx, ng = qp.nbu(n), qp.nbx(n), qp.ng(n)
        sel = []
        if which in ("u", "all"):
            sel += list(range(nbu))
        if which in ("x", "all"):
            sel += list(range(nbu, nbu + nbx))
        if which in ("g", "all"):
            sel += list(range(nbu + nbx, nbu + nbx + ng))
        m = len(sel)
        idxs[n] = np.array(sel, dtype=np.int32)
        Zl[n], Zu[n] = np.full(m, float(Z)), np.full(m, float(Z))
        zl[n], zu[n] = np.full(m, float(z)), np.full(m, float(z))
        lls[n], lus[n] = np.full(m, float(ls)), np.full(m, float(ls))
    new.idxs, new.Zl, new.Zu, new.zl, new.zu, new.lls, new.lus = idxs, Zl, Zu, zl, zu, lls, lus
    new.name = qp.name + f"_soft{which}"
    new.stage_key = [(k, "soft", which, float(Z), float(z), float(ls)) if n in set(stages) else k
                     for n, k in enumerate(qp.stage_key)] if qp.stage_key else []
    new.validate()
    return new


def perturb_x0(qp: OcpQp, x0_new: np.ndarray) -> OcpQp:
    """The same QP with the eliminated initial state replaced by ``x0_new``.
    Only stage-0 data depends on x0; it is rebuilt from the stage-1 model
    (A_1 = A, b_1 = b for these time-invariant workloads)."""
    import copy
    new = copy.copy(qp)
    for attr in ("b", "r", "lg", "ug"):
        setattr(new, attr, list(getattr(qp, attr)))
    A = qp.A[1]
    dx = x0_new - qp.x0
    new.b[0] = qp.b[0] + A @ dx
    new.r[0] = qp.r[0] + qp.S_full @ dx
    if qp.C0_full is not None:
        new.ug[0] = qp.ug[0] - qp.C0_full @ dx
        new.lg[0] = qp.lg[0] - qp.C0_full @ dx
    new.x0 = np.array(x0_new, dtype=np.float64)
    # stage 0 is new data: a key of its own, so that several perturbations of
    # one QP never alias in a shared-block batch
    new.stage_key = [(qp.name, "x0", np.asarray(x0_new, dtype=np.float64).tobytes())] + list(qp.stage_key[1:])
    return new
