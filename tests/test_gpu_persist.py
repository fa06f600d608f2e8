"""GPU parity of the one-launch RACE executors (RACE_EXEC_PERSIST_GROUP: one
leaf per lane group, plain updates of b; RACE_EXEC_PERSIST_CTA: one leaf per
block) and of the phase-by-phase executor with the transposed products off
the FP64 pipe
(RACE_EXEC_PHASE_DF64: one launch per phase over the leaves' rows in chunks)
against the CPU oracle, under the FP64 bound
|b_i - b_ref_i| <= 1e-12 sum_j |a_ij||x_j|.

Cases: fully recursed RACE schedules (many phases, the grid barrier between
each pair), one-level stage-0 groups, the MC and ABMC colourings (one phase
per colour), every lane-group width, FP32 values, SymmSpMM through the
phase executor, degenerate schedules (one phase, one row), two calls in a
row; and the grid barrier's timeout: a launch that expects one block too
many gives up at its first barrier, race_poll_status reports
RACE_ERR_TIMEOUT once, and the next call computes correctly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1907_06487_gb300 as R

pytestmark = pytest.mark.gpu

TOL = 1e-12
PG = R.RACE_EXEC_PERSIST_GROUP
PC = R.RACE_EXEC_PERSIST_CTA


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06487_gb300 import build
    build.build()
    return torch.device("cuda:0")


def use(s, exe, lanes=8):
    R.race_set_launch(s, 0, executor=exe, group_lanes=lanes, rows_per_group=1, blocks_per_sm=0, regs_per_row=4)


def run(s, x, dev):
    perm = s.perm()
    xd = torch.from_numpy(np.ascontiguousarray(x[perm])).to(dev)
    bd = torch.full_like(xd, np.nan)
    R.symm_spmv(s, xd, bd)
    torch.cuda.synchronize()
    R.race_poll_status(s)  # raises if a barrier gave up
    b = np.empty_like(x)
    b[perm] = bd.cpu().numpy()
    return b


def check(b, bref, sc):
    err = np.abs(b - bref)
    bound = TOL * sc + 1e-300
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), f"row {worst}: err {err[worst]:.3e} > {bound[worst]:.3e}"


MATS = {
    "st27": lambda g: g.stencil3d(16, npt=27, seed=2),
    "xxz": lambda g: g.xxz(16),
    "anderson": lambda g: g.anderson(18, W=16.5, seed=3),
    "geometric": lambda g: g.geometric(12000, seed=5, mean_degree=12.0),
}


@pytest.mark.parametrize("exe,lanes", [(PG, 4), (PG, 8), (PG, 32), (PG, 1), (PC, 8)])
@pytest.mark.parametrize("which", sorted(MATS))
def test_recursed_schedules(dev, oracle_mod, matgen_mod, which, exe, lanes):
    m = MATS[which](matgen_mod)
    s = R.race_build(m, 96, max_depth=-1, rcm=(which == "geometric"))
    sp, _, _ = s.phases()
    assert len(sp) - 1 >= 4  # several grid barriers
    use(s, exe, lanes)
    x = matgen_mod.uniform(m["n"], 17, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)
    check(run(s, x, dev), bref, sc)


@pytest.mark.parametrize("exe", [PG, PC])
def test_one_level_stage0(dev, oracle_mod, matgen_mod, exe):
    m = matgen_mod.xxz(18)
    s = R.race_build(m, 152, max_depth=-1, one_level_stage0=True)
    use(s, exe)
    x = matgen_mod.uniform(m["n"], 18, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)


@pytest.mark.parametrize("exe", [PG, PC])
@pytest.mark.parametrize("method,bs", [(R.RACE_COLOR_MC, 1), (R.RACE_COLOR_ABMC, 16)])
def test_colourings(dev, oracle_mod, matgen_mod, exe, method, bs):
    m = matgen_mod.stencil3d(12, npt=27, seed=4)
    s = R.race_build_coloring(m, method, bs)
    use(s, exe)
    x = matgen_mod.uniform(m["n"], 19, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)


@pytest.mark.parametrize("exe", [PG, PC])
def test_fp32_values(dev, oracle_mod, matgen_mod, exe):
    m = matgen_mod.stencil3d(14, npt=27, seed=6)
    m32 = dict(m, val=m["val"].astype(np.float32).astype(np.float64))
    s = R.race_build(m, 64, max_depth=-1, val_type=R.RACE_F32)
    use(s, exe)
    x = matgen_mod.uniform(m["n"], 20, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m32), x)
    check(run(s, x, dev), bref, sc)


@pytest.mark.parametrize("exe", [PG, PC])
def test_spmm_through_phases(dev, oracle_mod, matgen_mod, exe):
    m = matgen_mod.stencil3d(12, npt=27, seed=7)
    s = R.race_build(m, 64, max_depth=-1)
    use(s, exe)
    n, k = m["n"], 4
    X = matgen_mod.uniform(n * k, 21, -1.0, 1.0).reshape(n, k)
    Bref, S = oracle_mod.spmm_full(oracle_mod.expand_full(m), X)
    perm = s.perm()
    Xd = torch.from_numpy(np.ascontiguousarray(X[perm])).to(dev)
    Bd = torch.full_like(Xd, np.nan)
    R.symm_spmm(s, k, Xd, Bd)
    torch.cuda.synchronize()
    Bh = np.empty_like(X)
    Bh[perm] = Bd.cpu().numpy()
    check(Bh, Bref, S)


@pytest.mark.parametrize("exe", [PG, PC])
def test_degenerate(dev, oracle_mod, matgen_mod, exe):
    for m in (matgen_mod.banded(50, 1, seed=1, mean_degree=0.0), matgen_mod.banded(1, 1, seed=2, mean_degree=0.0),
              matgen_mod.stencil3d(6, npt=7, seed=3)):
        s = R.race_build(m, 1)  # one worker: one or two phases
        use(s, exe)
        x = matgen_mod.uniform(m["n"], 3)
        bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
        check(run(s, x, dev), bref, sc)


def test_barrier_timeout_is_reported(dev, oracle_mod, matgen_mod):
    m = matgen_mod.stencil3d(16, npt=27, seed=8)
    s = R.race_build(m, 96, max_depth=-1)
    n = m["n"]
    xd = torch.ones(n, dtype=torch.float64, device=dev)
    bd = torch.zeros_like(xd)
    R.race_probe_barrier_timeout(s, xd, bd)
    torch.cuda.synchronize()
    with pytest.raises(R.RaceError) as ei:
        R.race_poll_status(s)
    assert ei.value.code == R.RACE_ERR_TIMEOUT
    R.race_poll_status(s)  # cleared
    for exe in (PC, PG):   # the barrier words are reset by every launch
        use(s, exe)
        x = matgen_mod.uniform(n, 22, -1.0, 1.0)
        bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
        check(run(s, x, dev), bref, sc)
    one = R.race_build(matgen_mod.banded(1, 1, seed=1, mean_degree=0.0), 1)  # a single phase: no barrier
    assert len(one.phases()[0]) == 2
    with pytest.raises(R.RaceError) as ei:
        R.race_probe_barrier_timeout(one, xd[:1], bd[:1])
    assert ei.value.code == R.RACE_ERR_UNSUPPORTED


PD = R.RACE_EXEC_PHASE_DF64


@pytest.mark.parametrize("per_step,quarters", [(4, 2), (8, 1), (4, 0), (4, 4)])
@pytest.mark.parametrize("which", sorted(MATS))
def test_phase_df64(dev, oracle_mod, matgen_mod, which, per_step, quarters):
    # RACE_EXEC_DF64_RED's arithmetic phase by phase, the leaves' rows in chunks
    # of at most 256 rows: deep schedules (many phases, leaves of a few rows)
    # and depth-1 ones (few phases, leaves of thousands of rows)
    m = MATS[which](matgen_mod)
    x = matgen_mod.uniform(m["n"], 23, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    for depth in (-1, 1):
        s = R.race_build(m, 96, max_depth=depth, rcm=(which == "geometric"))
        R.race_set_launch(s, 0, executor=PD, group_lanes=1, rows_per_group=1, blocks_per_sm=0,
                          regs_per_row=per_step, fp64_quarters=quarters)
        check(run(s, x, dev), bref, sc)
        # by symm_spmv_exec while the schedule's launch names another executor
        R.race_set_launch(s, 0, executor=R.RACE_EXEC_ROWS_RED, group_lanes=2, rows_per_group=1, blocks_per_sm=0,
                          regs_per_row=8)
        perm = s.perm()
        xd = torch.from_numpy(np.ascontiguousarray(x[perm])).to(dev)
        bd = torch.full_like(xd, np.nan)
        R.symm_spmv_exec(s, PD, xd, bd)
        torch.cuda.synchronize()
        b = np.empty_like(x)
        b[perm] = bd.cpu().numpy()
        check(b, bref, sc)


def test_phase_df64_fp32_colourings_degenerate(dev, oracle_mod, matgen_mod):
    m = matgen_mod.stencil3d(13, npt=27, seed=9)
    m32 = dict(m, val=m["val"].astype(np.float32).astype(np.float64))
    x = matgen_mod.uniform(m["n"], 24, -1.0, 1.0)
    s = R.race_build(m, 64, max_depth=-1, val_type=R.RACE_F32)
    R.race_set_launch(s, 0, executor=PD, group_lanes=1, rows_per_group=1, blocks_per_sm=0, regs_per_row=4,
                      fp64_quarters=2)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m32), x)
    check(run(s, x, dev), bref, sc)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    for method, bs in ((R.RACE_COLOR_MC, 1), (R.RACE_COLOR_ABMC, 32)):
        c = R.race_build_coloring(m, method, bs)
        R.race_set_launch(c, 0, executor=PD, group_lanes=1, rows_per_group=1, blocks_per_sm=0, regs_per_row=4,
                          fp64_quarters=2)
        check(run(c, x, dev), bref, sc)
    for d in (matgen_mod.banded(1, 1, seed=2, mean_degree=0.0), matgen_mod.banded(300, 1, seed=1, mean_degree=0.0)):
        s = R.race_build(d, 4)
        R.race_set_launch(s, 0, executor=PD, group_lanes=1, rows_per_group=1, blocks_per_sm=0, regs_per_row=4)
        xx = matgen_mod.uniform(d["n"], 3)
        bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(d), xx)
        check(run(s, xx, dev), bref, sc)
