"""CPU tests of the library: it builds, loads, exports every declared symbol,
rejects malformed input, and its host-built schedules equal the oracle's
byte for byte (no GPU needed: RACE_FLAG_HOST_ONLY)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1907_06487_gb300 as R
from paper_1907_06487_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return R.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "race.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|int32_t|int64_t|void|char)\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(R.EXPORTED)


def test_strerror(lib):
    for code in range(0, 7):
        assert lib.race_strerror(code)
    assert b"unknown" in lib.race_strerror(99)


CASES = [
    ("paper16", lambda g: g.paper_stencil2d(16), 8, (0.6,), -1, 0),
    ("anderson10", lambda g: g.anderson(10, seed=1), 24, R.PAPER_EPS, -1, 0),
    ("anderson10_nnz", lambda g: g.anderson(10, seed=1), 24, R.PAPER_EPS, -1, 1),
    ("st27_10", lambda g: g.stencil3d(10, npt=27), 16, (0.5, 0.6, 0.5), 3, 0),
    ("geo", lambda g: g.geometric(4000, seed=11), 32, (0.7, 0.6, 0.5), -1, 0),
    ("xxz12", lambda g: g.xxz(12), 20, R.PAPER_EPS, -1, 0),
    ("band", lambda g: g.banded(2500, 90, seed=4), 10, (0.9, 0.8, 0.5), 2, 1),
]


@pytest.mark.parametrize("name,mk,nt,eps,md,bal", CASES, ids=[c[0] for c in CASES])
def test_host_schedule_matches_oracle(lib, oracle_mod, matgen_mod, name, mk, nt, eps, md, bal):
    m = mk(matgen_mod)
    s = R.race_build(m, nt, eps=eps, max_depth=md, balance=bal, host_only=True)
    o = oracle_mod.Race(m, nt, eps=eps, max_depth=md, balance=bal)
    assert s.export() == o.export()
    pm = oracle_mod.permute_upper(m, o.perm)
    lm = s.matrix()
    for k in ("row_ptr", "col", "val"):
        assert np.array_equal(pm[k], lm[k]), k
    info = s.info()
    assert info["eta"] == o.eta and info["n_phases"] == o.n_phases and info["n_leaves"] == o.n_leaves
    sp, lo, hi = s.phases()
    assert oracle_mod.check_phases(lm, sp, lo, hi) == 0


def test_noncanonical_input_is_canonicalised(lib, oracle_mod, matgen_mod):
    m = matgen_mod.anderson(6, seed=2)
    rng = np.random.default_rng(0)
    rp, col, val = m["row_ptr"], m["col"].copy(), m["val"].copy()
    # shuffle columns inside rows and drop every diagonal whose value we zero
    keep = np.ones(len(col), bool)
    for i in range(m["n"]):
        a, b = rp[i], rp[i + 1]
        p = rng.permutation(b - a) + a
        col[a:b], val[a:b] = col[p].copy(), val[p].copy()
        if i % 3 == 0:
            d = a + int(np.nonzero(col[a:b] == i)[0][0])
            keep[d] = False
    new_rp = np.concatenate([[0], np.cumsum([keep[rp[i]:rp[i + 1]].sum() for i in range(m["n"])])]).astype(np.int32)
    messy = {"n": m["n"], "row_ptr": new_rp, "col": col[keep], "val": val[keep]}
    canon = oracle_mod.canonicalize(messy)
    s = R.race_build(messy, 12, host_only=True)
    o = oracle_mod.Race(canon, 12)
    assert s.export() == o.export()
    lm = s.matrix()
    pm = oracle_mod.permute_upper(canon, o.perm)
    assert np.array_equal(lm["val"], pm["val"]) and np.array_equal(lm["col"], pm["col"])


def test_f32_values_keep_schedule(lib, oracle_mod, matgen_mod):
    m = matgen_mod.stencil3d(8, npt=27)
    s = R.race_build(m, 8, host_only=True, val_type=R.RACE_F32)
    o = oracle_mod.Race(m, 8)
    assert s.export() == o.export()
    lm = s.matrix()
    assert lm["val"].dtype == np.float32
    pm = oracle_mod.permute_upper(m, o.perm)
    assert np.array_equal(lm["val"], pm["val"].astype(np.float32))


def bad(m, **kw):
    with pytest.raises(R.RaceError) as e:
        R.race_build(m, kw.pop("nt", 4), host_only=True, **kw)
    return e.value.code


def test_rejects_malformed_input(lib):
    ok = {"n": 3, "row_ptr": np.array([0, 2, 3, 4], np.int32), "col": np.array([0, 1, 1, 2], np.int32),
          "val": np.array([1.0, 2.0, 3.0, 4.0])}
    R.race_build(ok, 2, host_only=True)
    below = dict(ok, col=np.array([0, 1, 0, 2], np.int32))
    assert bad(below) == R.RACE_ERR_INVALID
    dup = dict(ok, col=np.array([1, 1, 1, 2], np.int32))
    assert bad(dup) == R.RACE_ERR_INVALID
    oob = dict(ok, col=np.array([0, 3, 1, 2], np.int32))
    assert bad(oob) == R.RACE_ERR_INVALID
    nan = dict(ok, val=np.array([1.0, np.nan, 3.0, 4.0]))
    assert bad(nan) == R.RACE_ERR_INVALID
    inf = dict(ok, val=np.array([1.0, 2.0, np.inf, 4.0]))
    assert bad(inf) == R.RACE_ERR_INVALID
    nonmono = dict(ok, row_ptr=np.array([0, 3, 2, 4], np.int32))
    assert bad(nonmono) == R.RACE_ERR_INVALID
    assert bad(ok, nt=0) == R.RACE_ERR_INVALID
    assert bad(ok, eps=(0.4,)) == R.RACE_ERR_INVALID
    assert bad(ok, eps=(1.0,)) == R.RACE_ERR_INVALID
    assert bad(ok, group_lanes=3) == R.RACE_ERR_INVALID
    empty = {"n": 0, "row_ptr": np.array([0], np.int32), "col": np.zeros(0, np.int32), "val": np.zeros(0)}
    assert bad(empty) == R.RACE_ERR_INVALID
    # distance other than 2 is not built
    a = R.race_csr_upper(3, 4, ok["row_ptr"].ctypes.data, ok["col"].ctypes.data, ok["val"].ctypes.data, 0)
    p = R.make_params(2, host_only=True)
    p.dist_k = 1
    h = ctypes.c_void_p()
    assert lib.race_build(ctypes.byref(a), ctypes.byref(p), None, ctypes.byref(h)) == R.RACE_ERR_UNSUPPORTED
    assert b"distance" in lib.race_last_error_detail()


def test_host_only_schedule_refuses_compute(lib):
    m = {"n": 2, "row_ptr": np.array([0, 2, 3], np.int32), "col": np.array([0, 1, 1], np.int32),
         "val": np.array([2.0, 1.0, 2.0])}
    s = R.race_build(m, 1, host_only=True)
    with pytest.raises(R.RaceError) as e:
        R.symm_spmv(s, 0x1000, 0x2000)
    assert e.value.code == R.RACE_ERR_UNSUPPORTED
    # launch shapes are checked before anything else; the executor with the
    # transposed products off the FP64 pipe needs a device schedule
    for bad in (dict(fp64_quarters=5), dict(fp64_quarters=-1), dict(group_lanes=3), dict(executor=99)):
        with pytest.raises(R.RaceError) as e:
            R.race_set_launch(s, 0, **dict(dict(executor=R.RACE_EXEC_DF64_RED, group_lanes=1, rows_per_group=1), **bad))
        assert e.value.code == R.RACE_ERR_INVALID
    with pytest.raises(R.RaceError) as e:
        R.race_set_launch(s, 0, executor=R.RACE_EXEC_DF64_RED, group_lanes=1, rows_per_group=1)
    assert e.value.code == R.RACE_ERR_UNSUPPORTED
    s.free()
    with pytest.raises(RuntimeError):
        s.info()


def test_single_row_and_diagonal_only(lib, oracle_mod):
    one = {"n": 1, "row_ptr": np.array([0, 1], np.int32), "col": np.array([0], np.int32), "val": np.array([3.0])}
    s = R.race_build(one, 4, host_only=True)
    assert s.export() == oracle_mod.Race(one, 4).export()
    assert s.info()["n_leaves"] == 1
    n = 50
    diag = {"n": n, "row_ptr": np.arange(n + 1, dtype=np.int32), "col": np.arange(n, dtype=np.int32),
            "val": np.arange(1, n + 1, dtype=np.float64)}
    s = R.race_build(diag, 4, host_only=True)
    assert s.export() == oracle_mod.Race(diag, 4).export()


def test_natural_order_plan(matgen_mod):
    """RACE_FLAG_NATURAL_ORDER: identity permutation, the canonical input
    matrix unchanged, one phase with one leaf covering every row."""
    import paper_1907_06487_gb300 as R
    m = matgen_mod.anderson(6, seed=2)
    s = R.race_build(m, 8, host_only=True, natural_order=True)
    inf = s.info()
    assert inf["n_phases"] == 1 and inf["n_leaves"] == 1
    assert np.array_equal(s.perm(), np.arange(m["n"]))
    pm = s.matrix()
    for key in ("row_ptr", "col", "val"):
        assert np.array_equal(pm[key], m[key])
    sp, lo, hi = s.phases()
    assert list(sp) == [0, 1] and lo[0] == 0 and hi[0] == m["n"]


def test_rejects_sizes_beyond_the_int32_layout(lib):
    """Maximum sizes: the layout indexes rows and stored entries with int32, so
    n + nnz >= 2^31 is RACE_ERR_OVERFLOW (checked before any array is read:
    the arrays passed here are tiny placeholders)."""
    rp = np.zeros(4, np.int32)
    col = np.zeros(4, np.int32)
    val = np.zeros(4)
    p = R.make_params(4, host_only=True)
    h = ctypes.c_void_p()
    for n, nnz in ((3, 2 ** 31), (2 ** 30, 2 ** 30), (2 ** 31 - 1, 1)):
        a = R.race_csr_upper(n, nnz, rp.ctypes.data, col.ctypes.data, val.ctypes.data, 0)
        assert lib.race_build(ctypes.byref(a), ctypes.byref(p), None, ctypes.byref(h)) == R.RACE_ERR_OVERFLOW
        assert not h.value


@pytest.mark.parametrize("name", ["xxz26", "st27_200"])
def test_full_size_schedules_match_oracle(oracle_mod, name):
    """The benchmark's schedules at full size (XXZ L=26: 10.4 M rows; 27-point
    200^3: 8 M rows), built by the library on the host and by the oracle:
    identical byte images (permutation, phases, leaves, tree, eta)."""
    from paper_1907_06487_gb300 import configs
    m = configs.matrix(name)
    cfg = configs.SCHEDULE[name]
    s = R.race_build(m, cfg["n_workers"], eps=cfg["eps"], max_depth=cfg["max_depth"], host_only=True,
                     rcm=cfg.get("rcm", False))
    o = oracle_mod.Race(m, cfg["n_workers"], eps=cfg["eps"], max_depth=cfg["max_depth"], rcm=cfg.get("rcm", False))
    assert s.export() == o.export()
    s.free()


def test_noalloc_refuses_before_touching_the_device(lib):
    """symm_spmv_noalloc checks sizes, NULLs, aliasing and the 16-byte
    alignment its bulk copies need on the host, before any CUDA call (so the
    refusals need no GPU; the addresses below are never dereferenced)."""
    A = 0x10000  # 16-byte aligned stand-in addresses
    cases = [
        ((0, 0, A, A, A, A, A + 0x100), R.RACE_ERR_INVALID),            # n < 1
        ((8, 4, A, A, A, A, A + 0x100), R.RACE_ERR_INVALID),            # nnz < n
        ((8, 8, A, A, A, A, A), R.RACE_ERR_INVALID),                     # x and b alias
        ((8, 8, 0, A, A, A, A + 0x100), R.RACE_ERR_INVALID),             # NULL row_ptr
        ((8, 8, A + 4, A, A, A, A + 0x100), R.RACE_ERR_INVALID),         # row_ptr 4 bytes off
        ((8, 8, A, A + 8, A, A, A + 0x100), R.RACE_ERR_INVALID),         # col 8 bytes off
        ((8, 8, A, A, A + 8, A, A + 0x100), R.RACE_ERR_INVALID),         # val 8 bytes off
        (((1 << 24) + 1, (1 << 24) + 1, A, A, A, A, A + 0x100), R.RACE_ERR_OVERFLOW),
        ((8, (1 << 28) + 1, A, A, A, A, A + 0x100), R.RACE_ERR_OVERFLOW),
    ]
    for args, code in cases:
        with pytest.raises(R.RaceError) as e:
            R.symm_spmv_noalloc(*args)
        assert e.value.code == code, args
