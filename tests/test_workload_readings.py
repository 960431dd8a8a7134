"""Readings of the configured workloads, pinned on the CPU.

The mass-spring chain of Sec. 5.1 is configured as "Euler-discretised" with
dt = 0.5, |u| <= 0.5, |x| <= 4 over N = 30 stages.  The explicit (forward)
Euler step gives a model whose QPs have no feasible point, so the workload
uses the semi-implicit Euler step.  These tests make that reading checkable:
the two discretisations are rebuilt here from the continuous model, and a
linear program maximising the smallest constraint clearance shows every
explicit-Euler instance infeasible and every semi-implicit one feasible.
"""
import numpy as np
import pytest
from scipy.optimize import linprog

from paper_2003_02547_gb300 import workloads as W

M, DT, N = 8, 0.5, 30
UMAX, XMAX = 0.5, 4.0


def continuous_model():
    """pdot = v, vdot = T p + F u (unit masses and springs), T = tridiag(1, -2, 1)."""
    T = np.diag(-2.0 * np.ones(M)) + np.diag(np.ones(M - 1), 1) + np.diag(np.ones(M - 1), -1)
    F = np.zeros((M, M - 1))
    F[np.arange(M - 1), np.arange(M - 1)] = 1.0
    Ac = np.block([[np.zeros((M, M)), np.eye(M)], [T, np.zeros((M, M))]])
    Bc = np.vstack([np.zeros((M, M - 1)), F])
    return Ac, Bc, T, F


def clearance_lp(A, B, x0):
    """max m over u_0..u_{N-1}, m  s.t.  |u_n| <= UMAX - m, |x_n| <= XMAX - m
    (n = 1..N) along x_{n+1} = A x_n + B u_n; returns the optimal m."""
    nx, nu = B.shape
    nvar = N * nu + 1
    # x_n = A^n x0 + sum_k A^(n-1-k) B u_k : rows as affine maps of u
    rows, rhs = [], []
    Phi = [np.eye(nx)]
    for _ in range(N):
        Phi.append(A @ Phi[-1])
    for n in range(1, N + 1):
        G = np.zeros((nx, nvar))
        for k in range(n):
            G[:, k * nu:(k + 1) * nu] = Phi[n - 1 - k] @ B
        c = Phi[n] @ x0
        for s in (1.0, -1.0):
            row = s * G.copy()
            row[:, -1] = 1.0            # s x_n + m <= XMAX
            rows.append(row)
            rhs.append(XMAX - s * c)
    for k in range(N):
        for s in (1.0, -1.0):
            row = np.zeros((nu, nvar))
            row[:, k * nu:(k + 1) * nu] = s * np.eye(nu)
            row[:, -1] = 1.0            # s u_k + m <= UMAX
            rows.append(row)
            rhs.append(np.full(nu, UMAX))
    cost = np.zeros(nvar)
    cost[-1] = -1.0
    res = linprog(cost, A_ub=np.vstack(rows), b_ub=np.concatenate(rhs), bounds=[(None, None)] * (nvar - 1) + [(None, 1.0)],
                  method="highs")
    assert res.status == 0, res.message
    return -res.fun


def test_both_discretisations_follow_the_continuous_model():
    Ac, Bc, T, F = continuous_model()
    A_exp, B_exp = W.mass_spring_model(M, dt=DT, scheme="explicit")
    assert np.array_equal(A_exp, np.eye(2 * M) + DT * Ac)
    assert np.array_equal(B_exp, DT * Bc)
    # semi-implicit Euler: v+ = v + dt (T p + F u), p+ = p + dt v+
    A_si, B_si = W.mass_spring_model(M, dt=DT)
    rng = np.random.default_rng(7)
    for _ in range(5):
        p, v, u = rng.standard_normal(M), rng.standard_normal(M), rng.standard_normal(M - 1)
        v1 = v + DT * (T @ p + F @ u)
        p1 = p + DT * v1
        assert np.allclose(A_si @ np.concatenate([p, v]) + B_si @ u, np.concatenate([p1, v1]), atol=1e-13)
    # explicit Euler amplifies (spectral radius sqrt(1 + dt^2 * 4 sin^2) ~ 1.40);
    # the semi-implicit step keeps every mode on the unit circle, like the exact flow
    assert 1.39 < max(abs(np.linalg.eigvals(A_exp))) < 1.42
    assert np.allclose(abs(np.linalg.eigvals(A_si)), 1.0, atol=1e-9)


@pytest.mark.parametrize("index", [0, 1, 2, 3, 17, 511, 1023])
def test_explicit_euler_instances_are_infeasible_and_semi_implicit_feasible(index):
    qp = W.mass_spring_qp(index)
    x0 = qp.x0
    assert x0 is not None and np.all(np.abs(x0) <= 1.0)
    m_exp = clearance_lp(*W.mass_spring_model(M, dt=DT, scheme="explicit"), x0)
    m_si = clearance_lp(*W.mass_spring_model(M, dt=DT), x0)
    assert m_exp < 0.0, m_exp          # no point meets every bound
    assert m_si >= 0.4, m_si           # strictly feasible with a wide margin
