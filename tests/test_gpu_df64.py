"""GPU parity of the SymmSpMV executors that form the transposed updates off
the FP64 pipe, by an integer product of the significands (RACE_EXEC_DF64_RED
on the CRS, RACE_EXEC_SELL_DF64 on a SELL-32-sigma copy)
against the CPU oracle, under the FP64 bound
|b_i - b_ref_i| <= 1e-12 sum_j |a_ij||x_j|: every lane count, FP32 values,
entries per step of the SELL kernel, x entries that are zero or outside the
range [2^-50, 2^51) (those rows scatter in FP64), long rows on one lane, explicit zeros and large diagonal values, a
diagonal matrix and a single row, and the refusal of off-diagonal values
outside the range."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1907_06487_gb300 as R

pytestmark = pytest.mark.gpu

TOL = 1e-12
DF = R.RACE_EXEC_DF64_RED
SELL = R.RACE_EXEC_SELL_DF64
EXES = [DF, SELL]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06487_gb300 import build
    build.build()
    return torch.device("cuda:0")


def run(s, x, dev, executor=None):
    perm = s.perm()
    xd = torch.from_numpy(np.ascontiguousarray(x[perm])).to(dev)
    bd = torch.full_like(xd, np.nan)
    if executor is None:
        R.symm_spmv(s, xd, bd)
    else:
        R.symm_spmv_exec(s, executor, xd, bd)
    torch.cuda.synchronize()
    b = np.empty_like(x)
    b[perm] = bd.cpu().numpy()
    return b


def check(b, bref, sc):
    err = np.abs(b - bref)
    bound = TOL * sc + 1e-300
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), f"row {worst}: err {err[worst]:.3e} > {bound[worst]:.3e}"


@pytest.mark.parametrize("per_step", [4, 8])
@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_lanes(dev, oracle_mod, matgen_mod, lanes, per_step):
    m = matgen_mod.stencil3d(21, npt=27, seed=8)
    s = R.race_build(m, 32)
    R.race_set_launch(s, 0, executor=DF, group_lanes=lanes, rows_per_group=1, blocks_per_sm=0,
                      regs_per_row=per_step, fp64_quarters=1)
    x = matgen_mod.uniform(m["n"], 31, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)


@pytest.mark.parametrize("per_step", [4, 8, 16])
def test_sell_entries_per_step(dev, oracle_mod, matgen_mod, per_step):
    m = matgen_mod.xxz(16)  # rows of 1..9 upper entries: chunk tails of every length
    s = R.race_build(m, 32)
    R.race_set_launch(s, 0, executor=SELL, group_lanes=1, rows_per_group=1, blocks_per_sm=0, regs_per_row=per_step)
    x = matgen_mod.uniform(m["n"], 32, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)
    check(run(s, x, dev), bref, sc)


@pytest.mark.parametrize("exe", EXES)
def test_fp32_values(dev, oracle_mod, matgen_mod, exe):
    m = matgen_mod.xxz(16)
    m32 = dict(m, val=m["val"].astype(np.float32).astype(np.float64))
    s = R.race_build(m, 32, val_type=R.RACE_F32)
    x = matgen_mod.uniform(m["n"], 12)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m32), x)
    check(run(s, x, dev, exe), bref, sc)


@pytest.mark.parametrize("exe", EXES)
def test_x_outside_split_range_and_zeros(dev, oracle_mod, matgen_mod, exe):
    m = matgen_mod.anderson(20, W=16.5, seed=2)
    s = R.race_build(m, 32)
    n = m["n"]
    x = matgen_mod.uniform(n, 13, -1.0, 1.0)
    rng = np.random.default_rng(4)
    idx = rng.choice(n, 600, replace=False)
    x[idx[:200]] = 0.0
    x[idx[200:300]] = -0.0
    x[idx[300:400]] = 3.0e20     # above 2^51: FP64 entries
    x[idx[400:500]] = -7.0e-21   # below 2^-50
    x[idx[500:]] *= 2.0 ** 40    # inside the range, large
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev, exe), bref, sc)


@pytest.mark.parametrize("exe", EXES)
def test_long_rows_one_lane(dev, oracle_mod, matgen_mod, exe):
    m = matgen_mod.banded(3000, 700, seed=5, mean_degree=1000.0)  # ~500 upper entries per row
    s = R.race_build(m, 16)
    R.race_set_launch(s, 0, executor=exe, group_lanes=1, rows_per_group=1, blocks_per_sm=0, regs_per_row=4)
    x = matgen_mod.uniform(m["n"], 6, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)


def offdiag_index(m, k):
    rows = np.repeat(np.arange(m["n"]), np.diff(m["row_ptr"]))
    return np.flatnonzero(m["col"] != rows)[k]


@pytest.mark.parametrize("exe", EXES)
def test_explicit_zeros_and_large_diagonal(dev, oracle_mod, matgen_mod, exe):
    m = matgen_mod.anderson(16, W=16.5, seed=3)
    m = dict(m, val=m["val"].copy())
    rows = np.repeat(np.arange(m["n"]), np.diff(m["row_ptr"]))
    diag = np.flatnonzero(m["col"] == rows)
    m["val"][diag[::7]] = 1.0e30        # diagonal values need no split
    m["val"][diag[1::7]] = 0.0
    for k in range(0, 400, 3):
        m["val"][offdiag_index(m, k)] = 0.0  # explicit zeros scatter nothing
    s = R.race_build(m, 16)
    R.race_set_launch(s, 0, executor=exe, group_lanes=2, rows_per_group=1, blocks_per_sm=0, regs_per_row=4)
    x = matgen_mod.uniform(m["n"], 21, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)


@pytest.mark.parametrize("exe", EXES)
def test_values_out_of_range_refused(dev, matgen_mod, exe):
    m = matgen_mod.anderson(8, seed=1)
    m = dict(m, val=m["val"].copy())
    m["val"][offdiag_index(m, 3)] = 1.0e30
    s = R.race_build(m, 4)
    with pytest.raises(R.RaceError) as ei:
        R.race_set_launch(s, 0, executor=exe, group_lanes=1, rows_per_group=1, blocks_per_sm=0, regs_per_row=4)
    assert ei.value.code == R.RACE_ERR_UNSUPPORTED
    xd = torch.zeros(m["n"], dtype=torch.float64, device=dev)
    bd = torch.empty_like(xd)
    with pytest.raises(R.RaceError):
        R.symm_spmv_exec(s, exe, xd, bd)
    # the schedule still serves the FP64 executors
    R.symm_spmv_exec(s, R.RACE_EXEC_ROWS_RED, xd, bd)
    torch.cuda.synchronize()
    assert float(bd.abs().max()) == 0.0


@pytest.mark.parametrize("exe", EXES)
def test_degenerate(dev, oracle_mod, matgen_mod, exe):
    # diagonal only, a single row, zero x
    for m in (matgen_mod.banded(50, 1, seed=1, mean_degree=0.0), matgen_mod.banded(1, 1, seed=2, mean_degree=0.0)):
        s = R.race_build(m, 4)
        x = matgen_mod.uniform(m["n"], 3)
        bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
        check(run(s, x, dev, exe), bref, sc)
        z = np.zeros(m["n"])
        assert np.all(run(s, z, dev, exe) == 0.0)


@pytest.mark.parametrize("k", [2, 4, 8, 16])
@pytest.mark.parametrize("rows_in_flight", [1, 4])
@pytest.mark.parametrize("val_type", ["f64", "f32"])
def test_spmm_double_float_scatter(dev, oracle_mod, matgen_mod, k, rows_in_flight, val_type):
    m = matgen_mod.stencil3d(14, npt=27, seed=6)
    m = dict(m, val=m["val"].copy())
    rows = np.repeat(np.arange(m["n"]), np.diff(m["row_ptr"]))
    m["val"][np.flatnonzero(m["col"] != rows)[::11]] = 0.0  # explicit zeros scatter nothing
    vt = R.RACE_F64
    if val_type == "f32":
        m["val"] = m["val"].astype(np.float32).astype(np.float64)
        vt = R.RACE_F32
    s = R.race_build(m, 32, val_type=vt)
    R.race_set_launch(s, 0, executor=DF, group_lanes=1, rows_per_group=rows_in_flight, blocks_per_sm=0,
                      regs_per_row=4, fp64_quarters=1)
    n = m["n"]
    X = matgen_mod.uniform(n * k, 14, -1.0, 1.0).reshape(n, k)
    X[5, :] = 0.0
    X[7, 0] = 4.0e20        # outside the split's range: that column of row 7 scatters in FP64
    X[11, k - 1] = -3.0e-19
    Bref, S = oracle_mod.spmm_full(oracle_mod.expand_full(m), X)
    perm = s.perm()
    Xd = torch.from_numpy(np.ascontiguousarray(X[perm])).to(dev)
    Bd = torch.full_like(Xd, np.nan)
    R.symm_spmm(s, k, Xd, Bd)
    torch.cuda.synchronize()
    Bh = np.empty_like(X)
    Bh[perm] = Bd.cpu().numpy()
    check(Bh, Bref, S)


def test_probe_scatter(dev, matgen_mod):
    """race_probe_scatter: mode 0 adds 1 per stored off-diagonal entry to its
    column (the lower degree of every row), mode 1 stores the row's sum of
    column indices."""
    m = matgen_mod.xxz(12)
    s = R.race_build(m, 8)
    pm = s.matrix()
    n = pm["n"]
    rows = np.repeat(np.arange(n), np.diff(pm["row_ptr"]))
    off = pm["col"] != rows
    bd = torch.zeros(n, dtype=torch.float64, device=dev)
    R.race_probe_scatter(s, 0, bd)
    torch.cuda.synchronize()
    assert np.array_equal(bd.cpu().numpy(), np.bincount(pm["col"][off], minlength=n).astype(np.float64))
    R.race_probe_scatter(s, 1, bd)
    torch.cuda.synchronize()
    assert np.array_equal(bd.cpu().numpy(), np.bincount(rows, weights=pm["col"], minlength=n))
    with pytest.raises(R.RaceError):
        R.race_probe_scatter(s, 2, bd)


@pytest.mark.parametrize("exe", [R.RACE_EXEC_LEAF_GROUP, R.RACE_EXEC_ROWS_RED, DF, SELL])
def test_natural_order(dev, oracle_mod, matgen_mod, exe):
    """Without a RACE schedule (input order, one leaf) every executor still
    computes SymmSpMV; the leaf executor then runs the rows serially."""
    m = matgen_mod.xxz(12)
    s = R.race_build(m, 16, natural_order=True)
    x = matgen_mod.uniform(m["n"], 15, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev, exe), bref, sc)


@pytest.mark.parametrize("quarters", [0, 1, 2, 4])
def test_fp64_share_of_transposed_updates(dev, oracle_mod, matgen_mod, quarters):
    """fp64_quarters: that share of the warps forms its transposed updates with
    FP64 multiplies, the rest by the integer product; same bound either way (SpMV
    and SpMM, x with zeros and out-of-range entries)."""
    m = matgen_mod.stencil3d(15, npt=27, seed=9)
    s = R.race_build(m, 16)
    R.race_set_launch(s, 0, executor=DF, group_lanes=1, rows_per_group=1, blocks_per_sm=0, regs_per_row=4,
                      fp64_quarters=quarters)
    n = m["n"]
    x = matgen_mod.uniform(n, 19, -1.0, 1.0)
    x[::97] = 0.0
    x[5::101] = 1.0e25
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)
    k = 4
    X = matgen_mod.uniform(n * k, 20, -1.0, 1.0).reshape(n, k)
    X[3, 1] = -2.0e22
    Bref, S = oracle_mod.spmm_full(oracle_mod.expand_full(m), X)
    perm = s.perm()
    Xd = torch.from_numpy(np.ascontiguousarray(X[perm])).to(dev)
    Bd = torch.full_like(Xd, np.nan)
    R.symm_spmm(s, k, Xd, Bd)
    torch.cuda.synchronize()
    Bh = np.empty_like(X)
    Bh[perm] = Bd.cpu().numpy()
    check(Bh, Bref, S)
    with pytest.raises(R.RaceError):
        R.race_set_launch(s, 0, executor=DF, fp64_quarters=5)
