"""Synthetic workloads shaped like the paper's benchmark matrices.

Each workload is seeded and generated by ``matgen`` (the SuiteSparse/ScaMaC
matrices of the paper's Table "Details of the benchmark matrices" are not
available; these stand in for them):

  anderson32  3D Anderson model 32^3 periodic (7-pt, hopping -1, disorder
              U[-8.25, 8.25) seed 1), x ~ U[-1,1) seed 2   (paper: Anderson-16.5)
  xxz26       periodic Heisenberg XXZ chain L=26, Sz=0 (10,400,600 rows,
              J=1, Delta=1), x ~ U[-1,1) seed 3             (paper: Spin-26)
  st27_200    3D 27-pt stencil 200^3 nonperiodic, off-diag -U(0,1] seed 4,
              diag = row abs-sum + 1, X ~ U[-1,1) seed 5    (HPCG-like)

``SCHEDULE`` holds the schedule parameters the benchmark and the full-size
tests use for each workload.
"""
from __future__ import annotations

import numpy as np

from . import matgen

SEEDS = {"anderson32": (1, 2), "xxz26": (None, 3), "st27_200": (4, 5)}

# schedule parameters per workload: n_workers, eps, max_depth, the executor
# tested at full size, and the launch shapes of symm_spmv / spmv_full
# (shapes from the measured sweeps on GB300: one row per thread wins; FP64
# row sums with most transposed products formed on the integer pipes are
# faster than all-FP64 on every workload).  The recursion stops after stage 1 (two
# colours of level groups, Sec. 4.4.3): the executors that take the
# transposed update through L2 reductions use the schedule's permutation,
# not its phases, and the stage-0 level order keeps neighbours close while
# deeper sub-level orders scatter them (XXZ L=26: 0.34 ms at depth 1
# against 0.43 ms at unlimited depth; the 27-point stencil is indifferent).
# `rcm` relabels the matrix by reverse Cuthill-McKee first, as the paper
# does with all inputs (the 27-point stencil: 0.368 against 0.381 ms; XXZ
# and the lexicographic Anderson models unchanged, so they keep their order).
# The conflict-free executors need the full recursion's balance instead:
# `conflict_free` is the schedule they are measured on (the fastest of the
# measured N_t sweep that builds in seconds), with stage-0 groups of one
# level (upper storage keeps them write-disjoint; 27-point 100^3: 99 -> 63
# phases, leaf-per-CTA executor 0.996 -> 0.741 ms).  `sweeps` is the schedule
# of the Gauss-Seidel and Kaczmarz sweeps (distance-2 phases throughout: the
# Kaczmarz update writes every column of a row).
# (sweeps of blocks per SM x entries per step x FP64 share on GB300: XXZ L=26
# 6 blocks of 40-register threads, 4 entries; the 27-point stencil 4 blocks,
# 4 entries (0.372 ms at 8 entries per step).  With the transposed products
# formed by the integer product of the significands, a quarter of the row
# groups' products in FP64: XXZ 0.311 ms against 0.315 at share 0 and 0.321
# at 2/4; stencil 0.356 ms against 0.358 / 0.360)
_L = dict(executor=8, group_lanes=1, rows_per_group=1, blocks_per_sm=6, regs_per_row=4, fp64_quarters=1)
_LP = dict(executor=8, group_lanes=1, rows_per_group=1, blocks_per_sm=4, regs_per_row=4, fp64_quarters=1)
_F = dict(executor=2, group_lanes=1, rows_per_group=1, blocks_per_sm=4, regs_per_row=16)
SCHEDULE = {
    "anderson32": dict(n_workers=64, eps=(0.8, 0.8, 0.5), max_depth=-1, executor=1, launch=_L, full_launch=_F),
    "xxz26": dict(n_workers=152, eps=(0.8, 0.8, 0.5), max_depth=1, executor=1, launch=_L, full_launch=_F,
                  conflict_free=dict(n_workers=152, max_depth=-1, one_level_stage0=True)),
    "xxz24": dict(n_workers=152, eps=(0.8, 0.8, 0.5), max_depth=1, executor=1, launch=_L, full_launch=_F,
                  conflict_free=dict(n_workers=152, max_depth=-1, one_level_stage0=True)),
    "st27_200": dict(n_workers=152, eps=(0.8, 0.8, 0.5), max_depth=1, rcm=True, executor=1, launch=_LP,
                     full_launch=_F, conflict_free=dict(n_workers=2432, max_depth=-1, one_level_stage0=True),
                     sweeps=dict(n_workers=2432, max_depth=-1)),
    "st27_100": dict(n_workers=152, eps=(0.8, 0.8, 0.5), max_depth=1, rcm=True, executor=1, launch=_LP,
                     full_launch=_F, conflict_free=dict(n_workers=2432, max_depth=-1, one_level_stage0=True)),
}

# schedule of every matrix of the batch workload (same reasoning as above;
# the geometric graphs come in random point order, which the reverse
# Cuthill-McKee relabelling turns into neighbour-preserving order: 17-21 %
# faster SymmSpMV at 5e5-1e6 points)
BATCH_SCHEDULE = dict(n_workers=64, max_depth=1, rcm=True)


def batch64(count: int = 64, scale: float = 1.0) -> list:
    """The batch workload: alternately 3D Anderson models with L uniform in
    [16, 96] (disorder 16.5, per-matrix seed) and random geometric graphs with
    n uniform in [1e4, 1e6] points (unit cube, radius for mean degree 20,
    weights U(0,1], diag = sum + 1).  Draws from splitmix64 stream seed 6.
    `scale` < 1 shrinks every matrix (test-sized batches)."""
    u = matgen.uniform(2 * count, 6, 0.0, 1.0)
    out = []
    for i in range(count):
        if i % 2 == 0:
            L = 16 + int(u[i] * 81)
            L = max(4, int(round(L * scale ** (1.0 / 3.0))))
            out.append(dict(matgen.anderson(L, W=16.5, seed=100 + i), name=f"anderson{L}"))
        else:
            npts = 10000 + int(u[i] * (1000000 - 10000 + 1))
            npts = max(200, int(npts * scale))
            out.append(dict(matgen.geometric(npts, seed=200 + i), name=f"geometric{npts}"))
    return out


def matrix(name: str) -> dict:
    if name == "anderson32":
        return matgen.anderson(32, W=16.5, seed=1)
    if name == "xxz26":
        return matgen.xxz(26, J=1.0, Delta=1.0)
    if name == "st27_200":
        return matgen.stencil3d(200, npt=27, seed=4)
    if name.startswith("xxz"):
        return matgen.xxz(int(name[3:]))
    if name.startswith("anderson"):
        return matgen.anderson(int(name[8:]), W=16.5, seed=1)
    if name.startswith("st27_"):
        return matgen.stencil3d(int(name[5:]), npt=27, seed=4)
    raise KeyError(name)


def vectors(name: str, n: int, k: int = 1) -> np.ndarray:
    seed = SEEDS.get(name, (None, 7))[1]
    x = matgen.uniform(n * k, seed, -1.0, 1.0)
    return x if k == 1 else x.reshape(n, k)
