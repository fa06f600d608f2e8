"""GPU parity of the warp-tile staged SymmSpMV (RACE_EXEC_STAGED: values and
columns brought into shared memory by bulk copies, row sums in FP64 or
double-float and transposed products in FP64 or by the integer product of the
significands, per quarter of the warps) against the CPU
oracle, under the FP64 bound |b_i - b_ref_i| <= 1e-12 sum_j |a_ij||x_j|.

Cases: every mix of FP64 and double-float row sums with FP64 and integer
transposed products,
4 and 8 entries per lane and step, ragged last tiles, variable row lengths,
FP32-stored values, x entries that are zero or outside the split's range,
stored values outside it (taken in FP64, not refused), tiles too long to
stage and rows too long for a double-float sum, row sums that cancel below
the join's range, degenerate matrices, two calls in a row."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1907_06487_gb300 as R

pytestmark = pytest.mark.gpu

TOL = 1e-12
ST = R.RACE_EXEC_STAGED


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06487_gb300 import build
    build.build()
    return torch.device("cuda:0")


def staged(s, rs_q=0, tp_q=0, per_step=4, bps=0):
    R.race_set_launch(s, 0, executor=ST, group_lanes=1, rows_per_group=1, blocks_per_sm=bps,
                      regs_per_row=per_step, fp64_quarters=tp_q, rowsum_fp64_quarters=rs_q)


def run(s, x, dev):
    perm = s.perm()
    xd = torch.from_numpy(np.ascontiguousarray(x[perm])).to(dev)
    bd = torch.full_like(xd, np.nan)
    R.symm_spmv(s, xd, bd)
    torch.cuda.synchronize()
    R.race_poll_status(s)
    b = np.empty_like(x)
    b[perm] = bd.cpu().numpy()
    return b


def check(b, bref, sc):
    err = np.abs(b - bref)
    bound = TOL * sc + 1e-300
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), f"row {worst}: err {err[worst]:.3e} > {bound[worst]:.3e}"


@pytest.mark.parametrize("per_step", [4, 8])
@pytest.mark.parametrize("rs_q,tp_q", [(0, 0), (0, 4), (4, 0), (4, 4), (2, 2), (1, 3), (3, 1)])
def test_arithmetic_mixes(dev, oracle_mod, matgen_mod, rs_q, tp_q, per_step):
    m = matgen_mod.stencil3d(21, npt=27, seed=8)  # 9261 rows: 289 full tiles and a ragged one
    s = R.race_build(m, 32)
    staged(s, rs_q, tp_q, per_step)
    x = matgen_mod.uniform(m["n"], 31, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)


@pytest.mark.parametrize("bps", [1, 2])
def test_variable_rows_and_repeat(dev, oracle_mod, matgen_mod, bps):
    m = matgen_mod.xxz(16)  # rows of 1..9 upper entries
    s = R.race_build(m, 32)
    staged(s, 2, 2, 8, bps)
    x = matgen_mod.uniform(m["n"], 32, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)
    check(run(s, x, dev), bref, sc)


@pytest.mark.parametrize("rs_q", [0, 4])
def test_fp32_values(dev, oracle_mod, matgen_mod, rs_q):
    m = matgen_mod.stencil3d(17, npt=27, seed=3)
    m32 = dict(m, val=m["val"].astype(np.float32).astype(np.float64))
    s = R.race_build(m, 32, val_type=R.RACE_F32)
    staged(s, rs_q, 0)
    x = matgen_mod.uniform(m["n"], 12)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m32), x)
    check(run(s, x, dev), bref, sc)


@pytest.mark.parametrize("rs_q,tp_q", [(0, 0), (4, 0), (0, 4)])
def test_x_outside_split_range_and_zeros(dev, oracle_mod, matgen_mod, rs_q, tp_q):
    m = matgen_mod.anderson(20, W=16.5, seed=2)
    s = R.race_build(m, 32)
    staged(s, rs_q, tp_q)
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
    check(run(s, x, dev), bref, sc)


def test_values_outside_split_range_taken_in_fp64(dev, oracle_mod, matgen_mod):
    m = matgen_mod.anderson(16, W=16.5, seed=3)
    m = dict(m, val=m["val"].copy())
    rows = np.repeat(np.arange(m["n"]), np.diff(m["row_ptr"]))
    diag = np.flatnonzero(m["col"] == rows)
    off = np.flatnonzero(m["col"] != rows)
    m["val"][diag[::7]] = 1.0e30
    m["val"][diag[1::7]] = 0.0
    m["val"][off[::11]] = 3.0e-20      # below 2^-50
    m["val"][off[5::13]] = -2.0e17     # above 2^51
    m["val"][off[2::17]] = 0.0         # explicit zeros scatter nothing
    s = R.race_build(m, 16)
    x = matgen_mod.uniform(m["n"], 21, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    for rs_q, tp_q in ((0, 0), (2, 2), (4, 4)):
        staged(s, rs_q, tp_q)
        check(run(s, x, dev), bref, sc)


@pytest.mark.parametrize("rs_q", [0, 4])
def test_long_rows_and_unstaged_tiles(dev, oracle_mod, matgen_mod, rs_q):
    # ~500 upper entries per row: every tile exceeds the stage (read from
    # global memory) and every row exceeds the double-float row-sum length
    m = matgen_mod.banded(3000, 700, seed=5, mean_degree=1000.0)
    s = R.race_build(m, 16)
    staged(s, rs_q, 0)
    x = matgen_mod.uniform(m["n"], 6, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)


def test_mixed_stageable_tiles(dev, oracle_mod, matgen_mod):
    # rows of 2..60 entries: some tiles fit the stage, some do not; rows of
    # more than 64 entries nowhere, so every row sum runs in double-float
    m = matgen_mod.banded(5000, 120, seed=7, mean_degree=30.0)
    assert np.diff(m["row_ptr"]).max() <= 64
    s = R.race_build(m, 16, natural_order=True)
    staged(s, 0, 0, 8)
    x = matgen_mod.uniform(m["n"], 8, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)


def band2(n, diag, off):
    """Upper CRS: diagonal `diag`, coupling `off` to the next two rows."""
    rp = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n):
        for c, v in ((i, diag), (i + 1, off), (i + 2, off)):
            if c < n:
                cols.append(c)
                vals.append(v)
        rp[i + 1] = len(cols)
    return {"n": n, "row_ptr": rp, "col": np.array(cols, dtype=np.int32), "val": np.array(vals)}


def test_cancelling_row_sums(dev, oracle_mod):
    # diagonal 2^-40, couplings -2^-41 to the next two rows, and x = 2^-40
    # with every third entry 2^-40 (1 + 2^-30): the stored half of every row
    # but the last two sums to 2^-110 or -2^-111, below the range of the
    # integer join (binary exponent -102), so a double-float row sum takes
    # the FP64 conversion; with a constant x those sums cancel to zero
    n = 200
    m = band2(n, 2.0 ** -40, -(2.0 ** -41))
    s = R.race_build(m, 4, natural_order=True)
    for x in (2.0 ** -40 * (1.0 + (np.arange(n) % 3 == 0) * 2.0 ** -30), np.full(n, 2.0 ** -40)):
        bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
        for rs_q in (0, 4):
            staged(s, rs_q, 0)
            check(run(s, x, dev), bref, sc)


def test_degenerate(dev, oracle_mod, matgen_mod):
    # diagonal only, a single row, fewer rows than a tile, zero x
    for m in (matgen_mod.banded(50, 1, seed=1, mean_degree=0.0), matgen_mod.banded(1, 1, seed=2, mean_degree=0.0),
              matgen_mod.banded(7, 4, seed=3, mean_degree=3.0)):
        s = R.race_build(m, 4)
        staged(s, 0, 0)
        x = matgen_mod.uniform(m["n"], 3)
        bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
        check(run(s, x, dev), bref, sc)
        assert np.all(run(s, np.zeros(m["n"]), dev) == 0.0)


def test_launch_shape_refused_out_of_range(dev, matgen_mod):
    s = R.race_build(matgen_mod.anderson(8, seed=1), 4)
    with pytest.raises(R.RaceError):
        staged(s, 5, 0)
    with pytest.raises(R.RaceError):
        staged(s, 0, -1)


@pytest.mark.parametrize("stages", [1, 2])
def test_stage_count(dev, oracle_mod, matgen_mod, stages):
    m = matgen_mod.stencil3d(19, npt=27, seed=2)
    s = R.race_build(m, 16)
    R.race_set_launch(s, 0, executor=ST, group_lanes=1, rows_per_group=stages, blocks_per_sm=0, regs_per_row=4,
                      fp64_quarters=2, rowsum_fp64_quarters=4)
    x = matgen_mod.uniform(m["n"], 17, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)
    check(run(s, x, dev), bref, sc)


def test_bounded_wait_gives_up_and_reports(dev, oracle_mod, matgen_mod):
    """A wait that nothing completes (every mbarrier expects 16 bytes more than
    its copies deliver) gives up after its spin limit: the status word reads
    RACE_ERR_TIMEOUT exactly once, the context stays usable, and the next
    regular call is correct."""
    m = matgen_mod.stencil3d(15, npt=27, seed=4)
    s = R.race_build(m, 16)
    n = m["n"]
    x = matgen_mod.uniform(n, 9, -1.0, 1.0)
    xd = torch.from_numpy(x[s.perm()].copy()).to(dev)
    bd = torch.empty_like(xd)
    R.race_poll_status(s)  # clean before
    R.race_probe_wait_timeout(s, xd, bd)
    with pytest.raises(R.RaceError) as ei:
        R.race_poll_status(s)
    assert ei.value.code == R.RACE_ERR_TIMEOUT
    R.race_poll_status(s)  # cleared
    staged(s, 4, 4)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check(run(s, x, dev), bref, sc)
