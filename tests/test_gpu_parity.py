"""GPU parity: the device path (through the C ABI) against the CPU oracle.

Bound (FP64): |b_i - b_ref_i| <= 1e-12 * s_i with s_i = sum_j |a_ij||x_j|
from the oracle.  The kernels sum at most a row's worth of products in a
different order than the oracle, so their own error is below
nnz_row * 2^-53 * s_i (~1e-14 s_i here); 1e-12 is the required bound.
FP32-stored values are compared with the oracle applied to the FP32-rounded
matrix under the same bound (products and sums stay FP64).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1907_06487_gb300 as R
from paper_1907_06487_gb300 import configs

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06487_gb300 import build
    build.build()
    return torch.device("cuda:0")


def run_symm(s, m, x, dev, executor=None):
    perm = s.perm()
    xd = torch.from_numpy(np.ascontiguousarray(x[perm])).to(dev)
    bd = torch.empty_like(xd)
    if executor is None:
        R.symm_spmv(s, xd, bd)
    else:
        R.symm_spmv_exec(s, executor, xd, bd)
    torch.cuda.synchronize()
    b = np.empty_like(x)
    b[perm] = bd.cpu().numpy()
    return b


def assert_parity(b, bref, s, tol=TOL):
    err = np.abs(b - bref)
    bound = tol * s + 1e-300
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), f"row {worst}: err {err[worst]:.3e} > {bound[worst]:.3e}"


MATS = [
    ("paper16", lambda g: g.paper_stencil2d(16), 8, (0.6,), -1),
    ("anderson32", lambda g: g.anderson(32, W=16.5, seed=1), 64, R.PAPER_EPS, -1),
    ("anderson32_d1", lambda g: g.anderson(32, W=16.5, seed=1), 64, R.PAPER_EPS, 1),
    ("st27_24", lambda g: g.stencil3d(24, npt=27, seed=4), 48, R.PAPER_EPS, -1),
    ("xxz16", lambda g: g.xxz(16), 32, R.PAPER_EPS, -1),
    ("geo_islands", lambda g: g.geometric(30000, seed=12, mean_degree=6.0), 40, (0.6, 0.6, 0.5), -1),
    ("band", lambda g: g.banded(20000, 300, seed=3), 24, R.PAPER_EPS, -1),
    ("serial", lambda g: g.anderson(12, seed=5), 16, R.PAPER_EPS, 0),
    ("one_worker", lambda g: g.stencil3d(9, npt=7, seed=1), 1, R.PAPER_EPS, -1),
]


@pytest.mark.parametrize("executor", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9])
@pytest.mark.parametrize("name,mk,nt,eps,md", MATS, ids=[m[0] for m in MATS])
def test_symm_spmv_parity(dev, oracle_mod, matgen_mod, name, mk, nt, eps, md, executor):
    m = mk(matgen_mod)
    s = R.race_build(m, nt, eps=eps, max_depth=md)
    x = matgen_mod.uniform(m["n"], 77, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    assert_parity(run_symm(s, m, x, dev, executor), bref, sc)
    # second call on the same buffers overwrites, does not accumulate
    assert_parity(run_symm(s, m, x, dev, executor), bref, sc)


def test_default_entry_point(dev, oracle_mod, matgen_mod):
    m = matgen_mod.xxz(14)
    s = R.race_build(m, 16)
    x = matgen_mod.uniform(m["n"], 5)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    assert_parity(run_symm(s, m, x, dev), bref, sc)


@pytest.mark.parametrize("k", [1, 2, 4, 8, 16])
def test_symm_spmm_parity(dev, oracle_mod, matgen_mod, k):
    m = matgen_mod.stencil3d(20, npt=27, seed=4)
    s = R.race_build(m, 32)
    n = m["n"]
    X = matgen_mod.uniform(n * k, 5).reshape(n, k)
    Bref, S = oracle_mod.spmm_full(oracle_mod.expand_full(m), X)
    perm = s.perm()
    Xd = torch.from_numpy(np.ascontiguousarray(X[perm])).to(dev)
    Bd = torch.empty_like(Xd)
    R.symm_spmm(s, k, Xd, Bd)
    torch.cuda.synchronize()
    Bh = np.empty_like(X)
    Bh[perm] = Bd.cpu().numpy()
    assert_parity(Bh, Bref, S)


def test_fp32_values(dev, oracle_mod, matgen_mod):
    m = matgen_mod.stencil3d(22, npt=27, seed=4)
    m32 = dict(m, val=m["val"].astype(np.float32).astype(np.float64))
    s = R.race_build(m, 32, val_type=R.RACE_F32)
    x = matgen_mod.uniform(m["n"], 9)
    bref32, sc32 = oracle_mod.spmv_full(oracle_mod.expand_full(m32), x)
    b = run_symm(s, m, x, dev)
    assert_parity(b, bref32, sc32)
    bref64, sc64 = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    normwise = np.linalg.norm(b - bref64) / np.linalg.norm(sc64)
    assert normwise <= 2.0 ** -24


def test_spmv_full_parity(dev, oracle_mod, matgen_mod):
    for m in (matgen_mod.xxz(16), matgen_mod.anderson(20, seed=3), matgen_mod.stencil3d(16, npt=27)):
        s = R.race_build(m, 32)
        x = matgen_mod.uniform(m["n"], 3)
        perm = s.perm()
        xd = torch.from_numpy(np.ascontiguousarray(x[perm])).to(dev)
        bd = torch.empty_like(xd)
        R.spmv_full(s, xd, bd)
        torch.cuda.synchronize()
        b = np.empty_like(x)
        b[perm] = bd.cpu().numpy()
        bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
        assert_parity(b, bref, sc)


def test_permute_roundtrip(dev, matgen_mod):
    m = matgen_mod.anderson(10, seed=2)
    s = R.race_build(m, 16)
    perm = s.perm()
    for k in (1, 3):
        X = matgen_mod.uniform(m["n"] * k, 4).reshape(m["n"], k)
        Xd = torch.from_numpy(X).to(dev)
        Pd = torch.empty_like(Xd)
        Ud = torch.empty_like(Xd)
        R.race_permute(s, Xd, Pd, k)
        R.race_unpermute(s, Pd, Ud, k)
        torch.cuda.synchronize()
        assert np.array_equal(Pd.cpu().numpy(), X[perm])
        assert np.array_equal(Ud.cpu().numpy(), X)


def test_rejects_aliasing_and_bad_k(dev, matgen_mod):
    m = matgen_mod.anderson(6, seed=2)
    s = R.race_build(m, 4)
    x = torch.zeros(m["n"], dtype=torch.float64, device=dev)
    with pytest.raises(R.RaceError):
        R.symm_spmv(s, x, x)
    with pytest.raises(R.RaceError):
        R.symm_spmm(s, 3, x, torch.zeros_like(x))
    with pytest.raises(R.RaceError):
        R.symm_spmm(s, 17, x, torch.zeros_like(x))


# ---- full-size workloads in the benchmark's launch configuration ------------------------------

def sample_rows(n, perm_bounds, count, seed):
    rng = np.random.default_rng(seed)
    rows = set(rng.choice(n, size=min(count, n), replace=False).tolist())
    rows.update([0, n - 1])
    rows.update(int(v) for v in perm_bounds if 0 <= v < n)
    return np.array(sorted(rows), np.int32)


def test_full_size_xxz26(dev, oracle_mod):
    name = "xxz26"
    m = configs.matrix(name)
    cfg = configs.SCHEDULE[name]
    s = R.race_build(m, cfg["n_workers"], eps=cfg["eps"], max_depth=cfg["max_depth"], rcm=cfg.get("rcm", False))
    n = m["n"]
    x = configs.vectors(name, n)
    perm = s.perm()
    # rows at leaf boundaries (original numbering) plus a random sample
    sp, lo, hi = s.phases()
    rows = sample_rows(n, perm[np.concatenate([lo, hi - 1])][:2000], 3000, 1)
    bref, sc = oracle_mod.spmv_sampled(m, x, rows)
    # the launch the benchmark times (through the default entry point), then
    # the leaf executors
    lc = cfg["launch"]
    R.race_set_launch(s, 0, **lc)
    assert_parity(run_symm(s, m, x, dev)[rows], bref, sc)
    for ex in (cfg["executor"], 0, R.RACE_EXEC_PERSIST_CTA, R.RACE_EXEC_PERSIST_GROUP):
        b = run_symm(s, m, x, dev, ex)
        R.race_poll_status(s)  # no grid barrier gave up
        assert_parity(b[rows], bref, sc)
    # property at every row: the uniform vector is an eigenvector, eigenvalue L/4 = 6.5,
    # and every partial sum is a multiple of 1/4 (exact in FP64, and in the
    # integer products: 0.5 * 1 has a short significand, so truncation is exact)
    ones = np.ones(n)
    assert np.all(run_symm(s, m, ones, dev) == 6.5)
    b1 = run_symm(s, m, ones, dev, cfg["executor"])
    assert np.all(b1 == 6.5)
    assert np.all(run_symm(s, m, ones, dev, R.RACE_EXEC_PERSIST_CTA) == 6.5)


_ST27 = {}


def st27_schedule():
    if not _ST27:
        name = "st27_200"
        m = configs.matrix(name)
        cfg = configs.SCHEDULE[name]
        _ST27["m"] = m
        _ST27["s"] = R.race_build(m, cfg["n_workers"], eps=cfg["eps"], max_depth=cfg["max_depth"],
                                  rcm=cfg.get("rcm", False))
        lc = cfg["launch"]  # the launch the benchmark times
        R.race_set_launch(_ST27["s"], 0, **lc)
    return _ST27["m"], _ST27["s"]


@pytest.mark.parametrize("k", [1, 4, 8, 16])
def test_full_size_st27_200_spmm(dev, oracle_mod, k):
    name = "st27_200"
    m, s = st27_schedule()
    n = m["n"]
    X = configs.vectors(name, n, k)
    perm = s.perm()
    rows = sample_rows(n, [], 1500, 2)
    Bref, S = oracle_mod.spmv_sampled(m, X if k > 1 else X.reshape(n), rows)
    Xd = torch.from_numpy(np.ascontiguousarray(X[perm])).to(dev)
    Bd = torch.empty_like(Xd)
    if k == 1:
        R.symm_spmv(s, Xd, Bd)
    else:
        R.symm_spmm(s, k, Xd, Bd)
    torch.cuda.synchronize()
    Bh = np.empty_like(X)
    Bh[perm] = Bd.cpu().numpy()
    assert_parity(Bh[rows].reshape(Bref.shape), Bref, S)
