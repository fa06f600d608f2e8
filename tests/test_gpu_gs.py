"""GPU parity of symm_gs and symm_kacz (symmetric Gauss-Seidel and symmetric
Kaczmarz under a RACE schedule, through the C ABI) against the oracle's
orc_symm_gs and orc_symm_kacz on the same schedule.

The matrices are diagonally dominant (diagonal = row abs sum + 1), so a sweep
is contractive: a rounding difference in one row (the kernel sums a row in
another order than the oracle) shrinks by sum|a_ij| / |a_ii| < 1 in the rows
that read it.  Bound per row: |x - x_ref| <= 1e-12 (sum_{j != i} |a_ij|
|x_ref_j| + |b_i|) / |a_ii|, the row update's own magnitude.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1907_06487_gb300 as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06487_gb300 import build
    build.build()
    return torch.device("cuda:0")


def dense_scale(full, x, b):
    n = full["n"]
    rows = np.repeat(np.arange(n), np.diff(full["row_ptr"]))
    off = full["col"] != rows
    acc = np.zeros(n)
    np.add.at(acc, rows[off], np.abs(full["val"][off]) * np.abs(x[full["col"][off]]))
    d = np.zeros(n)
    np.add.at(d, rows[~off], full["val"][~off])
    return (acc + np.abs(b)) / np.abs(d)


CASES = [
    ("st27_16_full", lambda g: g.stencil3d(16, npt=27, seed=4), 48, {}),
    ("st27_16_one_level", lambda g: g.stencil3d(16, npt=27, seed=4), 48, {"max_depth": 1, "one_level_stage0": True}),
    ("geo_islands_rcm", lambda g: g.geometric(20000, seed=12, mean_degree=6.0), 40, {"rcm": True}),
    ("band", lambda g: g.banded(5000, 80, seed=2), 24, {}),
    ("st27_12_f32", lambda g: g.stencil3d(12, npt=27, seed=7), 32, {"val_type": R.RACE_F32}),
]


@pytest.mark.parametrize("name,mk,nt,kw", CASES, ids=[c[0] for c in CASES])
def test_symm_gs_parity(dev, oracle_mod, matgen_mod, name, mk, nt, kw):
    m = mk(matgen_mod)
    s = R.race_build(m, nt, **kw)
    full = oracle_mod.expand_full(s.matrix())  # the library's permuted matrix (values as stored)
    sp, lo, hi = s.phases()
    n = m["n"]
    rng = np.random.default_rng(11)
    b, x0 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    want = oracle_mod.symm_gs(full, sp, lo, hi, b, x0, 2)
    bd = torch.from_numpy(b).to(dev)
    xd = torch.from_numpy(x0.copy()).to(dev)
    R.symm_gs(s, bd, xd, 2)
    torch.cuda.synchronize()
    got = xd.cpu().numpy()
    bound = 1e-12 * dense_scale(full, want, b)
    worst = int(np.argmax(np.abs(got - want) / bound))
    assert np.all(np.abs(got - want) <= bound), f"row {worst}: {abs(got[worst] - want[worst]):.3e} > {bound[worst]:.3e}"


def test_symm_gs_edges(dev, matgen_mod):
    m = matgen_mod.stencil3d(8, npt=7, seed=1)
    s = R.race_build(m, 16)
    n = m["n"]
    b = torch.ones(n, dtype=torch.float64, device=dev)
    x = torch.full((n,), 0.25, dtype=torch.float64, device=dev)
    R.symm_gs(s, b, x, 0)  # no sweep: x unchanged
    torch.cuda.synchronize()
    assert torch.all(x == 0.25)
    for bad in ((b, b, 1), (b, x, -1)):
        with pytest.raises(R.RaceError) as e:
            R.symm_gs(s, *bad)
        assert e.value.code == R.RACE_ERR_INVALID
    h = R.race_build(m, 16, host_only=True)
    with pytest.raises(R.RaceError) as e:
        R.symm_gs(h, b, x, 1)
    assert e.value.code == R.RACE_ERR_UNSUPPORTED


# Kaczmarz writes every column of a row: the one-level stage-0 schedule
# (write-disjoint for half storage only) is refused instead (below)
KACZ_CASES = [c for c in CASES if "one_level" not in c[0]] + [("anderson12", lambda g: g.anderson(12, seed=1), 48, {})]


@pytest.mark.parametrize("name,mk,nt,kw", KACZ_CASES, ids=[c[0] for c in KACZ_CASES])
def test_symm_kacz_parity(dev, oracle_mod, matgen_mod, name, mk, nt, kw):
    """symm_kacz against the oracle, entry by entry.  Row projections are
    nonexpansive, so a rounding difference (another summation order of a.x and
    |a|^2) is not amplified by later rows; entry j only moves through the
    projections of the rows that contain it, which read its neighbours.  So
    each entry is held to 1e-12 of its local scale: the largest |x0_k| +
    |x_k| over j and its neighbours k in the full matrix."""
    m = mk(matgen_mod)
    s = R.race_build(m, nt, **kw)
    full = oracle_mod.expand_full(s.matrix())
    sp, lo, hi = s.phases()
    n = m["n"]
    rng = np.random.default_rng(13)
    b, x0 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    want = oracle_mod.symm_kacz(full, sp, lo, hi, b, x0, 2)
    bd = torch.from_numpy(b).to(dev)
    xd = torch.from_numpy(x0.copy()).to(dev)
    R.symm_kacz(s, bd, xd, 2)
    torch.cuda.synchronize()
    got = xd.cpu().numpy()
    mag = np.abs(want) + np.abs(x0)
    frp, fcol = full["row_ptr"], full["col"]
    local = np.maximum.reduceat(mag[fcol], frp[:-1]) if len(fcol) else mag
    local = np.maximum(local, mag)
    err = np.abs(got - want)
    worst = int(np.argmax(err / local))
    assert np.all(err <= 1e-12 * local), f"entry {worst}: {err[worst]:.3e} > 1e-12 * {local[worst]:.3e}"
    with pytest.raises(R.RaceError):
        R.symm_kacz(s, bd, bd, 1)


def test_symm_kacz_refuses_one_level_stage0(dev, matgen_mod):
    m = matgen_mod.stencil3d(16, npt=27, seed=4)
    s = R.race_build(m, 48, max_depth=1, one_level_stage0=True)
    b = torch.ones(m["n"], dtype=torch.float64, device=dev)
    x = torch.zeros_like(b)
    with pytest.raises(R.RaceError) as e:
        R.symm_kacz(s, b, x, 1)
    assert e.value.code == R.RACE_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.all(x == 0.0)  # nothing ran
    R.symm_gs(s, b, x, 1)  # Gauss-Seidel needs distance 1 only: accepted


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("sched", ["race", "mc", "abmc8"])
def test_sweeps_every_lane_count(dev, oracle_mod, matgen_mod, sched, lanes):
    """Both sweeps with every lane-group width, on a RACE schedule (leaves of
    many rows: the rows of a leaf one after the other) and on the MC and ABMC
    colourings (leaves of one and of 8 rows), against the oracle on the same
    schedule; rows of up to 27 entries span one or several steps of four
    entries a lane."""
    m = matgen_mod.stencil3d(12, npt=27, seed=5)
    if sched == "race":
        s = R.race_build(m, 32, max_depth=-1)
    elif sched == "mc":
        s = R.race_build_coloring(m, R.RACE_COLOR_MC, 1)
    else:
        s = R.race_build_coloring(m, R.RACE_COLOR_ABMC, 8)
    R.race_set_launch(s, 0, executor=R.RACE_EXEC_LEAF_GROUP, group_lanes=lanes, rows_per_group=1, blocks_per_sm=0,
                      regs_per_row=8)
    full = oracle_mod.expand_full(s.matrix())
    sp, lo, hi = s.phases()
    n = m["n"]
    rng = np.random.default_rng(17)
    b, x0 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    bd = torch.from_numpy(b).to(dev)
    want = oracle_mod.symm_gs(full, sp, lo, hi, b, x0, 2)
    xd = torch.from_numpy(x0.copy()).to(dev)
    R.symm_gs(s, bd, xd, 2)
    torch.cuda.synchronize()
    got = xd.cpu().numpy()
    bound = 1e-12 * dense_scale(full, want, b)
    assert np.all(np.abs(got - want) <= bound), float(np.max(np.abs(got - want) / bound))
    want = oracle_mod.symm_kacz(full, sp, lo, hi, b, x0, 2)
    xd = torch.from_numpy(x0.copy()).to(dev)
    R.symm_kacz(s, bd, xd, 2)
    torch.cuda.synchronize()
    got = xd.cpu().numpy()
    mag = np.abs(want) + np.abs(x0)
    local = np.maximum(np.maximum.reduceat(mag[full["col"]], full["row_ptr"][:-1]), mag)
    assert np.all(np.abs(got - want) <= 1e-12 * local), float(np.max(np.abs(got - want) / local))
