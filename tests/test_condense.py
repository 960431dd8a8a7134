"""Partial condensing (Sec. 3.5) through the C ABI, checked with the oracle
on the CPU: the condensed QP, read back from the staged data and solved by
the oracle, expands to a point that meets the original QP's KKT conditions
and equals the oracle's solution of the original QP."""
import numpy as np
import pytest

from oracle import ocp_ipm as O
from paper_2003_02547_gb300 import condense as CD
from paper_2003_02547_gb300 import workloads as W
from paper_2003_02547_gb300.batch import QpBatch


@pytest.fixture(scope="module")
def built():
    from paper_2003_02547_gb300 import build
    build.build()


CASES = [("mass-spring", lambda: W.mass_spring_qp(2, N=12)),
         ("small", lambda: W.small_random_qp(3)),
         ("ragged", lambda: W.ragged_random_qp(4, N_range=(9, 9), nx_range=(6, 6)))]


@pytest.mark.parametrize("block", [2, 3, 5])
@pytest.mark.parametrize("name,make", CASES)
def test_condensed_qp_expands_to_the_original_solution(built, name, make, block):
    qp = make()
    src = QpBatch([qp], device=None)
    dims = CD.condensed_dims(src, 0, block)
    assert dims[0] == -(-qp.N // block)
    dst = CD.condense(src, [0], block, device=None)
    cqp = dst.to_ocp(0)
    assert cqp.N == dims[0]
    rc = O.solve(cqp)
    assert rc.status == O.CONVERGED, name
    y, pi, lam, t = CD.expand(src, 0, block, dst, 0, sol=(rc.y, rc.pi, rc.lam, rc.t))
    kkt = O.full_residuals(qp, y, pi, lam, t)
    assert max(kkt[:4]) <= 1e-8, (name, block, kkt)
    ref = O.solve(qp)
    assert ref.status == O.CONVERGED
    err = np.max(np.abs(y - ref.y)) / max(1.0, np.max(np.abs(ref.y)))
    assert err <= 1e-6, (name, block, err)


def test_block_one_is_the_same_qp(built):
    qp = W.small_random_qp(1)
    src = QpBatch([qp], device=None)
    dst = CD.condense(src, [0], 1, device=None)
    cqp = dst.to_ocp(0)
    for n in range(qp.N + 1):
        np.testing.assert_allclose(cqp.Q[n], qp.Q[n], atol=1e-15)
        np.testing.assert_allclose(cqp.R[n], qp.R[n], atol=1e-15)
        if n < qp.N:
            np.testing.assert_allclose(cqp.A[n], qp.A[n], atol=1e-15)
            np.testing.assert_allclose(cqp.B[n], qp.B[n], atol=1e-15)
