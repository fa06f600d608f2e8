"""GPU checks of race_import and of the RACE_FLAG_PSEUDO_PERIPHERAL, RACE_FLAG_RCM and
RACE_FLAG_ONE_LEVEL_STAGE0 schedules through the C
ABI: an imported device schedule computes bit for bit what the schedule it
was exported from computes with the deterministic phase executor (a leaf per
lane group, plain updates of b in a fixed order), and both kinds of schedule
meet the parity bound |b_i - b_ref_i| <= 1e-12 s_i against the oracle's
plain definition with the phase executor and the default executor."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1907_06487_gb300 as R

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06487_gb300 import build
    build.build()
    return torch.device("cuda:0")


def run(s, x, dev, executor):
    perm = s.perm()
    xd = torch.from_numpy(np.ascontiguousarray(x[perm])).to(dev)
    bd = torch.empty_like(xd)
    R.symm_spmv_exec(s, executor, xd, bd)
    torch.cuda.synchronize()
    b = np.empty_like(x)
    b[perm] = bd.cpu().numpy()
    return b


def assert_parity(b, bref, sc):
    err = np.abs(b - bref)
    bound = TOL * sc + 1e-300
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), f"row {worst}: err {err[worst]:.3e} > {bound[worst]:.3e}"


CASES = [
    ("anderson24", lambda g: g.anderson(24, seed=1), 64, -1),
    ("xxz16_d1", lambda g: g.xxz(16), 152, 1),
    ("geo_islands", lambda g: g.geometric(30000, seed=12, mean_degree=6.0), 40, -1),
]


@pytest.mark.parametrize("name,mk,nt,md", CASES, ids=[c[0] for c in CASES])
def test_imported_schedule_runs_identically(dev, oracle_mod, matgen_mod, name, mk, nt, md):
    m = mk(matgen_mod)
    s = R.race_build(m, nt, max_depth=md)
    t = R.race_import(m, s.export())
    assert t.export() == s.export()
    x = matgen_mod.uniform(m["n"], 41, -1.0, 1.0)
    b_s = run(s, x, dev, R.RACE_EXEC_LEAF_GROUP)
    b_t = run(t, x, dev, R.RACE_EXEC_LEAF_GROUP)
    assert np.array_equal(b_s, b_t)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    assert_parity(b_t, bref, sc)
    assert_parity(run(t, x, dev, R.RACE_EXEC_DF64_RED), bref, sc)


def test_import_of_a_host_built_image_uploads(dev, oracle_mod, matgen_mod):
    """Schedules built on the host (no GPU needed) and imported on the
    device: the cache path for schedules prepared elsewhere."""
    m = matgen_mod.stencil3d(16, npt=27, seed=4)
    img = R.race_build(m, 48, host_only=True).export()
    t = R.race_import(m, img)
    x = matgen_mod.uniform(m["n"], 42, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    assert_parity(run(t, x, dev, R.RACE_EXEC_LEAF_GROUP), bref, sc)
    assert_parity(run(t, x, dev, R.RACE_EXEC_DF64_RED), bref, sc)


@pytest.mark.parametrize("name,mk,nt,md", CASES, ids=[c[0] for c in CASES])
def test_pseudo_peripheral_schedule_parity(dev, oracle_mod, matgen_mod, name, mk, nt, md):
    m = mk(matgen_mod)
    s = R.race_build(m, nt, max_depth=md, pseudo_peripheral=True)
    assert s.export() == oracle_mod.Race(m, nt, max_depth=md, pseudo_peripheral=True).export()
    x = matgen_mod.uniform(m["n"], 43, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    for executor in (R.RACE_EXEC_LEAF_GROUP, R.RACE_EXEC_DF64_RED):
        assert_parity(run(s, x, dev, executor), bref, sc)


@pytest.mark.parametrize("name,mk,nt,md", CASES, ids=[c[0] for c in CASES])
def test_rcm_schedule_parity(dev, oracle_mod, matgen_mod, name, mk, nt, md):
    """Schedules built on the reverse Cuthill-McKee relabelled matrix
    (RACE_FLAG_RCM): equal to the oracle's, parity-green with the phase
    executor and the default executor."""
    m = mk(matgen_mod)
    s = R.race_build(m, nt, max_depth=md, rcm=True)
    assert s.export() == oracle_mod.Race(m, nt, max_depth=md, rcm=True).export()
    x = matgen_mod.uniform(m["n"], 44, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    for executor in (R.RACE_EXEC_LEAF_GROUP, R.RACE_EXEC_DF64_RED):
        assert_parity(run(s, x, dev, executor), bref, sc)


@pytest.mark.parametrize("name,mk,nt,md", CASES, ids=[c[0] for c in CASES])
def test_one_level_stage0_parity(dev, oracle_mod, matgen_mod, name, mk, nt, md):
    """Stage-0 groups of one level (RACE_FLAG_ONE_LEVEL_STAGE0): the phase
    executors, which update b with plain stores inside a leaf (0), with
    reductions inside a leaf (1) and through shared-memory windows flushed
    with plain stores (7), stay parity-green on them."""
    m = mk(matgen_mod)
    s = R.race_build(m, nt, max_depth=md, one_level_stage0=True)
    assert s.export() == oracle_mod.Race(m, nt, max_depth=md, one_level_stage0=True).export()
    x = matgen_mod.uniform(m["n"], 45, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    for executor in (R.RACE_EXEC_LEAF_GROUP, R.RACE_EXEC_LEAF_CTA, R.RACE_EXEC_WINDOW_RACE, R.RACE_EXEC_DF64_RED):
        assert_parity(run(s, x, dev, executor), bref, sc)
