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
