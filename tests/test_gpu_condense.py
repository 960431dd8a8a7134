"""Partially condensed QPs solved on the GPU and expanded back (GPU)."""
import numpy as np
import pytest

import test_gpu_parity as GP
from test_gpu_parity import env  # noqa: F401  (shared module fixture)
from oracle import ocp_ipm as O
from paper_2003_02547_gb300 import condense as CD
from paper_2003_02547_gb300 import workloads as W
from paper_2003_02547_gb300.batch import QpBatch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("block", [2, 3])
def test_condensed_batch_solves_and_expands(env, block):
    gq, _, torch = env
    qps = [W.mass_spring_qp(i) for i in range(4)] + [W.ragged_random_qp(i) for i in range(2)]
    src = QpBatch(qps, device=None)
    for prec in (1, 0):
        dst = CD.condense(src, range(len(qps)), block)
        dst.upload()
        dst.solve(gq.default_arg(0, prec))
        dst.download()
        torch.cuda.synchronize()
        st = dst.all_stats()
        assert np.all(st["status"] == 0), st
        for i, qp in enumerate(qps):
            y, pi, lam, t = CD.expand(src, i, block, dst, i)
            kkt = O.full_residuals(qp, y, pi, lam, t)
            assert max(kkt[:4]) <= GP.KKT_TOL * 1.01, (i, prec, kkt)
            if i in (0, 4):
                ref = O.solve(qp)
                if ref.status == O.CONVERGED:
                    assert GP.rel_err(y, ref.y) <= GP.EXACT_TOL, (i, GP.rel_err(y, ref.y))


def _getters(b, i):
    """All staged data of QP i of batch b through the C getters."""
    import ctypes
    lib = b.lib
    out = []
    dims = b.stage_dims(i)
    for n, (nx, nu, nbx, nbu, ng) in enumerate(dims):
        nx1 = dims[n + 1][0] if n + 1 < len(dims) else 0
        P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        Pi = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        A, B, bb = np.zeros((max(1, nx1), max(1, nx)), order="F"), np.zeros((max(1, nx1), max(1, nu)), order="F"), \
            np.zeros(max(1, nx1))
        if n < len(dims) - 1:
            assert lib.gq_get_dynamics(b.h, i, n, P(A), max(1, nx1), P(B), max(1, nx1), P(bb)) == 0
        Q, S, R = np.zeros((max(1, nx), max(1, nx)), order="F"), np.zeros((max(1, nu), max(1, nx)), order="F"), \
            np.zeros((max(1, nu), max(1, nu)), order="F")
        q, r = np.zeros(max(1, nx)), np.zeros(max(1, nu))
        assert lib.gq_get_cost(b.h, i, n, P(Q), max(1, nx), P(S), max(1, nu), P(R), max(1, nu), P(q), P(r)) == 0
        iu, lu, uu = np.zeros(max(1, nbu), np.int32), np.zeros(max(1, nbu)), np.zeros(max(1, nbu))
        ix, lx, ux = np.zeros(max(1, nbx), np.int32), np.zeros(max(1, nbx)), np.zeros(max(1, nbx))
        assert lib.gq_get_box(b.h, i, n, Pi(iu), P(lu), P(uu), Pi(ix), P(lx), P(ux)) == 0
        C, Dm = np.zeros((max(1, ng), max(1, nx)), order="F"), np.zeros((max(1, ng), max(1, nu)), order="F")
        lg, ug = np.zeros(max(1, ng)), np.zeros(max(1, ng))
        assert lib.gq_get_general(b.h, i, n, P(C), max(1, ng), P(Dm), max(1, ng), P(lg), P(ug)) == 0
        out.append(dict(A=A, B=B, b=bb, Q=Q, S=S, R=R, q=q, r=r, iu=iu, lu=lu, uu=uu, ix=ix, lx=lx, ux=ux, C=C, D=Dm,
                        lg=lg, ug=ug))
    return out


@pytest.mark.parametrize("block", [2, 5])
def test_device_condensing_matches_host_condensing(env, block):
    """The condensing kernel writes the same condensed QPs as the host
    condensing (both the backward recursion of Sec. 3.5): equal data to
    rounding, identical box indices and masked sides."""
    gq, _, torch = env
    qps = [W.mass_spring_qp(i) for i in range(3)] + [W.ragged_random_qp(i) for i in (16, 31)] + \
        [W.small_random_qp(1)]
    src = QpBatch(qps)
    src.upload()
    dev = CD.condense_device(src, block)
    host = CD.condense(QpBatch(qps, device=None), range(len(qps)), block, device=None)
    for i in range(len(qps)):
        for n, (g, h) in enumerate(zip(_getters(dev, i), _getters(host, i))):
            for key in h:
                a, e = g[key], h[key]
                if a.dtype.kind == "i":
                    assert np.array_equal(a, e), (i, n, key)
                else:
                    fin = np.isfinite(e)
                    assert np.array_equal(fin, np.isfinite(a)) and np.array_equal(a[~fin], e[~fin]), (i, n, key)
                    scale = max(1.0, float(np.max(np.abs(e[fin]), initial=0.0)))
                    assert np.max(np.abs(a[fin] - e[fin]), initial=0.0) <= 1e-12 * scale, (i, n, key)


@pytest.mark.parametrize("block", [2, 3])
def test_device_condensed_solutions_match_the_oracle(env, block):
    """Device-condensed batch solved on the GPU and expanded: FP64 against the
    oracle solving the same condensed QP with the same exit rule (same
    trajectory, 1e-6 in y after expansion), both precisions within 1e-6 of
    the original QP's optimum when both sides run to complementarity 1e-14."""
    gq, _, torch = env
    import test_gpu_optimum as GO
    qps = [W.mass_spring_qp(i) for i in range(3)] + [W.ragged_random_qp(i) for i in (16, 31)]
    src = QpBatch(qps)
    src.upload()
    dst = CD.condense_device(src, block)
    for prec in (0, 1):
        dst.upload_sol()
        dst.solve(gq.default_arg(0, prec))
        dst.download()
        torch.cuda.synchronize()
        assert np.all(dst.all_stats()["status"] == 0), dst.all_stats()
        for i, qp in enumerate(qps):
            y, pi, lam, t = CD.expand(src, i, block, dst, i)
            kkt = O.full_residuals(qp, y, pi, lam, t)
            assert max(kkt[:4]) <= GP.KKT_TOL * 1.01, (i, prec, kkt)
            if prec == 0:
                cq = dst.to_ocp(i)
                same = O.solve(cq, O.IpmArg(**GP.SAME_RULE))
                assert same.status == O.CONVERGED
                ye = CD.expand(src, i, block, dst, i, sol=(same.y, same.pi, same.lam, same.t))[0]
                assert GP.rel_err(y, ye) <= GP.SOL_TOL, (i, GP.rel_err(y, ye))
        dst.upload_sol()
        dst.solve(gq.default_arg(0, prec, **GO.GPU_OPT_RULE))
        dst.download()
        torch.cuda.synchronize()
        assert np.all(dst.all_stats()["status"] == 0), dst.all_stats()
        for i, qp in enumerate(qps):
            y = CD.expand(src, i, block, dst, i)[0]
            opt = O.solve(qp, O.IpmArg(**GO.OPT_RULE))
            assert opt.status == O.CONVERGED
            assert GP.rel_err(y, opt.y) <= GO.OPT_TOL, (i, prec, GP.rel_err(y, opt.y))
