"""Planted mistakes in the oracle must be caught by its pins.

Each case patches one plausible error into the CPU oracle (a dropped term, a
flipped sign, a transposed block) and checks that at least one pin of
test_oracle_pins fails.  Nothing here touches a GPU.
"""
import numpy as np
import pytest

import test_oracle_pins as P
from oracle import ocp_ipm as O

_orig_assemble = O.assemble
_orig_step = O.KktFactor.step


def _mut_assemble(kind):
    def f(qp):
        dq = _orig_assemble(qp)
        if kind == "b_sign":
            dq.b = -dq.b
        elif kind == "drop_S":
            for n in range(qp.N + 1):
                o, nu, nx = dq.var_off[n], qp.nu[n], qp.nx[n]
                dq.H[o:o + nu, o + nu:o + nu + nx] = 0.0
                dq.H[o + nu:o + nu + nx, o:o + nu] = 0.0
        elif kind == "S_swapped":
            # S placed below the diagonal as S instead of S^T (square S only)
            for n in range(qp.N + 1):
                o, nu, nx = dq.var_off[n], qp.nu[n], qp.nx[n]
                if nu == nx and nu:
                    blk = dq.H[o:o + nu, o + nu:o + nu + nx].copy()
                    dq.H[o + nu:o + nu + nx, o:o + nu] = blk
        elif kind == "A_transposed":
            for n in range(qp.N):
                if qp.nx[n] == qp.nx[n + 1] and qp.nx[n]:
                    rows = slice(dq.eq_off[n], dq.eq_off[n + 1])
                    o, nu, nx = dq.var_off[n], qp.nu[n], qp.nx[n]
                    dq.A[rows, o + nu:o + nu + nx] = -qp.A[n].T
        elif kind == "upper_bound_sign":
            full = np.zeros(dq.nside)
            full[dq.active] = dq.d
            for n in range(qp.N + 1):
                c = (dq.side_off[n + 1] - dq.side_off[n]) // 2
                s = dq.side_off[n] + c
                full[s:s + c] = -full[s:s + c]
            dq.d = full[dq.active]
        return dq
    return f


def _mut_soft(kind):
    """Planted mistakes in the slack (soft-constraint) terms of the assembly."""
    def f(qp):
        dq = _orig_assemble(qp)
        act_idx = np.cumsum(dq.active) - 1          # full side -> row of dq.C
        for n in range(qp.N + 1):
            m = qp.ns(n)
            if not m:
                continue
            o = dq.var_off[n] + qp.nu[n] + qp.nx[n]
            c = qp.nbu(n) + qp.nbx(n) + qp.ng(n)
            s = dq.side_off[n]
            for k in range(m):
                jl, ju = o + k, o + m + k
                if kind == "drop_Z":
                    dq.H[jl, jl] = dq.H[ju, ju] = 0.0
                elif kind == "drop_z":
                    dq.g[jl] = dq.g[ju] = 0.0
                elif kind == "slack_upper_sign":
                    full = s + c + int(qp.idxs[n][k])
                    if dq.active[full]:
                        dq.C[act_idx[full], ju] = -1.0
        return dq
    return f


def _soft_pins():
    import test_oracle_soft as S
    S.test_scalar_soft_bound_closed_form("lower", 4.0, 0.5)
    S.test_scalar_soft_bound_closed_form("upper", 10.0, 2.0)
    for seed in range(6):
        S.test_soft_brute_force_active_sets(seed)


def _mut_step(kind):
    def step(self, rg, rb, rd, rm):
        dq, lam, t = self.dq, self.lam, self.t
        W = lam / t
        if kind == "gtilde_sign":
            gt = rg + dq.C.T @ (W * rd - rm / t)
        else:
            gt = rg - dq.C.T @ (W * rd - rm / t)
        sol = self.solve_reduced(-np.concatenate([gt, rb]))
        dy, dpi = sol[:dq.ny], sol[dq.ny:]
        dt = dq.C @ dy - rd
        if kind == "dlam_sign":
            dlam = (rm + lam * dt) / t
        else:
            dlam = -(rm + lam * dt) / t
        return dy, dpi, dlam, dt
    return step


def _square_lq(seed):
    return P.random_lq(seed, N=4, nxs=[2] * 5, nus=[2] * 4 + [0])


def _pins_fail(checks):
    failed = 0
    for fn in checks:
        try:
            fn()
        except (AssertionError, np.linalg.LinAlgError):
            failed += 1
    return failed


def _lqr_pin_square():
    qp = _square_lq(3)
    res = O.solve(qp)
    assert res.status == O.CONVERGED
    us, xs, pis = P.riccati_dp(qp)
    st = O.split_stages(qp, res.dq, res.y)
    for n in range(qp.N + 1):
        np.testing.assert_allclose(st[n][0], us[n], rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(st[n][1], xs[n], rtol=1e-9, atol=1e-10)


def _brute_pins():
    for seed in range(4):
        P.test_brute_force_active_sets(seed)


@pytest.mark.parametrize("kind", ["b_sign", "drop_S", "S_swapped", "A_transposed",
                                  "upper_bound_sign"])
def test_planted_assembly_mistake_is_caught(monkeypatch, kind):
    monkeypatch.setattr(O, "assemble", _mut_assemble(kind))
    checks = [P.test_unconstrained_matches_riccati_dp, _lqr_pin_square, _brute_pins]
    assert _pins_fail(checks) >= 1, kind


@pytest.mark.parametrize("kind", ["gtilde_sign", "dlam_sign"])
def test_planted_newton_mistake_is_caught(monkeypatch, kind):
    monkeypatch.setattr(O.KktFactor, "step", _mut_step(kind))
    checks = [P.test_reduced_newton_step_equals_full_system, _brute_pins]
    assert _pins_fail(checks) >= 1, kind


@pytest.mark.parametrize("kind", ["drop_Z", "drop_z", "slack_upper_sign"])
def test_planted_slack_mistake_is_caught(monkeypatch, kind):
    monkeypatch.setattr(O, "assemble", _mut_soft(kind))
    assert _pins_fail([_soft_pins]) >= 1, kind


def test_unmutated_oracle_passes_the_soft_checks():
    assert _pins_fail([_soft_pins]) == 0


def test_unmutated_oracle_passes_the_same_checks():
    checks = [P.test_unconstrained_matches_riccati_dp, _lqr_pin_square, _brute_pins,
              P.test_reduced_newton_step_equals_full_system]
    assert _pins_fail(checks) == 0
