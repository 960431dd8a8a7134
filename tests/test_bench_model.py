"""The flop model behind bench.py's roofline, checked on the CPU.

The roofline divides algorithmic flops by the kernel time and compares them
with a flop-mix peak in which each class of work runs on the unit that does
it: FP32 factorisations and solves on the FP32 lanes, FP64 ones on the FP64
pipe, and the one-warp kernel's double-float residual mat-vecs on the FP32
lanes at DF_COST instructions per multiply-add.  These tests fix the per-QP
counts against a hand count and the attribution of each class.
"""
import numpy as np

import bench
from paper_2003_02547_gb300 import workloads as W

STATS = np.dtype([("n_fact", "<i4"), ("n_fact64", "<i4"), ("n_solve", "<i4"), ("n_res", "<i4")])


def stats(nf, nf64, ns, nr):
    return np.array([(nf, nf64, ns, nr)], dtype=STATS)[0]


def test_per_qp_counts_by_hand():
    qp = W.small_random_qp(0, N=3, nx=2, nu=1)
    f, s, r = bench.qp_flops(qp)
    # stage sizes of this QP: x0 is eliminated (stage 0 has nu = 1, nx = 0),
    # the terminal stage has no input; (nv, nx_{n+1}) per stage
    sizes = [(1, 2), (3, 2), (3, 2), (2, 0)]
    f_hand = sum(m * m * v + m * v * v + v ** 3 / 3.0 for v, m in sizes)
    s_hand = sum(2.0 * (v * v + 2.0 * m * v) for v, m in sizes)
    assert [qp.nx[n] + qp.nu[n] for n in range(4)] == [v for v, _ in sizes]
    assert np.isclose(f, f_hand) and s == s_hand
    assert r == s_hand  # no general rows: a residual costs what a solve does


def test_split_of_a_one_warp_qp():
    qp = W.mass_spring_qp(0)
    f, s, r = bench.qp_flops(qp)
    # all factorisations in FP32: residuals are double-float, nothing in FP64
    f32, f64, fdf = bench.work_split([qp], [stats(7, 0, 22, 23)])
    assert (f32, f64, fdf) == (7 * f + 22 * s, 0.0, 23 * r)
    # half the factorisations in FP64 (a hand-over): solves and residuals split alike
    f32, f64, fdf = bench.work_split([qp], [stats(8, 4, 20, 20)])
    assert np.isclose(f32, 4 * f + 10 * s) and np.isclose(f64, 4 * f + 10 * s + 10 * r) and np.isclose(fdf, 10 * r)
    # the same QP forced into the block kernel: its residuals are FP64
    f32, f64, fdf = bench.work_split([qp], [stats(7, 0, 22, 23)], warp_max_nv=0)
    assert fdf == 0.0 and f64 == 23 * r


def test_block_kernel_qp_residuals_are_fp64():
    qp = W.large_stage_qp(0, N=3)
    f, s, r = bench.qp_flops(qp)
    f32, f64, fdf = bench.work_split([qp], [stats(6, 0, 20, 21)])
    assert fdf == 0.0 and f64 == 21 * r and f32 == 6 * f + 20 * s


def test_t_min_weights_each_class_by_its_unit():
    saved = dict(bench.PEAKS)
    try:
        bench.PEAKS.update(fp32=80e12, fp64=1e12)
        assert np.isclose(bench.t_min_of(80e12, 0.0, 0.0), 1.0)
        assert np.isclose(bench.t_min_of(0.0, 1e12, 0.0), 1.0)
        assert np.isclose(bench.t_min_of(0.0, 0.0, 80e12), bench.DF_COST)
    finally:
        bench.PEAKS.clear()
        bench.PEAKS.update(saved)
