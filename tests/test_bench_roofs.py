"""The roofline arithmetic and labels of bench.py on CPU: SymmSpMM's bound
min(HBM x intensity, FP64 roof) with the FP64 roof set by the row sums'
multiply-adds alone, the plain all-FP64 roof beside it, which bound wins on
either side of the crossover, and the arithmetic and dtype labels of the
executors.  The figures are the 27-point 200^3 stencil's (8,000,000 rows,
110,923,596 stored upper and 213,847,192 full entries)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1907_06487_gb300 import perfmodel as pm  # noqa: E402

N, NU, NF = 8_000_000, 110_923_596, 213_847_192
HBM, DFMA = 6779.4, 0.526e12


@pytest.mark.parametrize("k", [4, 8, 16])
def test_spmm_roof_fp64_floor(k):
    flops, nbytes = pm.flops(NF, k), pm.symm_bytes_rmw(N, NU, k)
    # a kernel exactly at the row sums' FP64 floor: nnz_u * k multiply-adds at the measured rate
    t_floor = NU * k / DFMA
    r = bench.spmm_roof(flops, nbytes, t_floor, HBM, DFMA, NU * k)
    assert r["intensity_flop_per_byte"] == pytest.approx(flops / nbytes)
    # 2 nnz_f / nnz_u flops per multiply-add: just under 4 for a stencil with its diagonal
    assert r["roof_gflops"] == pytest.approx(2 * NF / NU * DFMA / 1e9)
    assert r["bound"] == "fp64" and r["frac_of_roof"] == pytest.approx(1.0)
    # the all-FP64 form: every flop on the FP64 pipe, 2 per multiply-add
    assert r["plain_fp64_roof_gflops"] == pytest.approx(2 * DFMA / 1e9)
    assert r["frac_of_plain_fp64_roof"] == pytest.approx(NF / NU)
    assert r["frac_hbm"] == pytest.approx(nbytes / t_floor / 1e9 / HBM)


def test_spmm_roof_hbm_side():
    # k = 1: 0.275 flop per byte puts the HBM roof (1.86 TFLOP/s) below the
    # row sums' FP64 floor (2.03 TFLOP/s); the fraction is then bytes / time / bandwidth
    flops, nbytes = pm.flops(NF, 1), pm.symm_bytes_rmw(N, NU, 1)
    t = 0.35e-3
    r = bench.spmm_roof(flops, nbytes, t, HBM, DFMA, NU)
    assert r["bound"] == "hbm"
    assert r["frac_of_roof"] == pytest.approx(r["frac_hbm"])
    assert r["roof_gflops"] == pytest.approx(HBM * flops / nbytes)
    # at k = 4 the FP64 floor binds
    assert bench.spmm_roof(pm.flops(NF, 4), pm.symm_bytes_rmw(N, NU, 4), t, HBM, DFMA, 4 * NU)["bound"] == "fp64"


def test_labels():
    head = dict(executor=8, group_lanes=1, rows_per_group=1, blocks_per_sm=6, regs_per_row=4, fp64_quarters=1)
    a = bench.arithmetic_label(head)
    assert "1/4" in a and "3/4" in a and "integer" in a
    assert bench.dtype_label(head) == "f64"
    assert bench.dtype_label(dict(head, executor=13)) == "f64"
    assert bench.arithmetic_label(dict(executor=3)) == "f64" and bench.dtype_label(dict(executor=3)) == "f64"
    staged = dict(executor=10, fp64_quarters=2, rowsum_fp64_quarters=1)
    assert bench.dtype_label(staged) == "f64+df64"
    assert "double-float" in bench.arithmetic_label(staged)
    assert bench.dtype_label(dict(staged, rowsum_fp64_quarters=4)) == "f64"
