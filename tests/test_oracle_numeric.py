"""Pins of the oracle's numeric part against things other than itself.

Each test checks the oracle (``oracle/race_oracle.c``) against dense linear
algebra (numpy), exact integer arithmetic, or closed forms of the synthetic
matrices; a dropped transpose term, a wrong index or a sign error in the
oracle fails at least one of them.
"""
import math

import numpy as np
import pytest


def random_upper(n, density, seed, with_diag=True, ints=False):
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        if with_diag:
            rows.append(i); cols.append(i); vals.append(float(rng.integers(-5, 6)) if ints else rng.normal())
        for j in range(i + 1, n):
            if rng.random() < density:
                rows.append(i); cols.append(j); vals.append(float(rng.integers(-5, 6)) if ints else rng.normal())
    rows, cols, vals = np.array(rows), np.array(cols, np.int32), np.array(vals)
    rp = np.zeros(n + 1, np.int32)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    return {"n": n, "row_ptr": rp, "col": cols, "val": vals}


def dense_of(m):
    n = m["n"]
    A = np.zeros((n, n))
    for i in range(n):
        for t in range(m["row_ptr"][i], m["row_ptr"][i + 1]):
            j = m["col"][t]
            A[i, j] = m["val"][t]
            A[j, i] = m["val"][t]
    return A


@pytest.mark.parametrize("n,density,seed", [(1, 0.0, 0), (7, 0.5, 1), (40, 0.2, 2), (120, 0.05, 3)])
def test_full_spmv_matches_dense(oracle_mod, n, density, seed):
    m = random_upper(n, density, seed)
    A = dense_of(m)
    x = np.random.default_rng(seed + 100).uniform(-1, 1, n)
    full = oracle_mod.expand_full(m)
    b, s = oracle_mod.spmv_full(full, x)
    np.testing.assert_allclose(b, A @ x, rtol=0, atol=1e-13 * max(1.0, np.abs(A).sum()))
    np.testing.assert_allclose(s, np.abs(A) @ np.abs(x), rtol=1e-14)


def test_full_expansion_is_exact_transpose(oracle_mod):
    m = random_upper(60, 0.15, 5)
    full = oracle_mod.expand_full(m)
    n = full["n"]
    D = np.zeros((n, n))
    for i in range(n):
        for t in range(full["row_ptr"][i], full["row_ptr"][i + 1]):
            D[i, full["col"][t]] = full["val"][t]
        cols = full["col"][full["row_ptr"][i]:full["row_ptr"][i + 1]]
        assert np.all(np.diff(cols) > 0)
    assert np.array_equal(D, D.T)
    assert np.array_equal(D, dense_of(m))


def test_integer_matrix_exact(oracle_mod):
    # integer entries and integer x: every partial sum is an exact double
    m = random_upper(80, 0.2, 7, ints=True)
    A = dense_of(m)
    x = np.random.default_rng(8).integers(-9, 10, 80).astype(np.float64)
    exact = (A.astype(np.int64) @ x.astype(np.int64)).astype(np.float64)
    b, _ = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    assert np.array_equal(b, exact)
    assert np.array_equal(oracle_mod.symm_spmv(m, x), exact)
    bs, _ = oracle_mod.spmv_sampled(m, x, np.arange(80))
    assert np.array_equal(bs, exact)


def test_serial_symm_spmv_matches_dense(oracle_mod):
    m = random_upper(150, 0.06, 9)
    x = np.random.default_rng(10).uniform(-1, 1, 150)
    np.testing.assert_allclose(oracle_mod.symm_spmv(m, x), dense_of(m) @ x, rtol=0, atol=1e-12)


def test_sampled_rows_match_dense(oracle_mod):
    m = random_upper(90, 0.1, 11)
    A = dense_of(m)
    X = np.random.default_rng(12).uniform(-1, 1, (90, 4))
    rows = np.array([0, 5, 89, 44, 13], np.int32)
    B, S = oracle_mod.spmv_sampled(m, X, rows)
    np.testing.assert_allclose(B, (A @ X)[rows], rtol=0, atol=1e-12)
    np.testing.assert_allclose(S, (np.abs(A) @ np.abs(X))[rows], rtol=1e-13)
    with pytest.raises(ValueError):
        oracle_mod.spmv_sampled(m, X, np.array([3, 3], np.int32))


def test_spmm_columns_match_dense(oracle_mod):
    m = random_upper(70, 0.1, 13)
    A = dense_of(m)
    X = np.random.default_rng(14).uniform(-1, 1, (70, 8))
    B, S = oracle_mod.spmm_full(oracle_mod.expand_full(m), X)
    np.testing.assert_allclose(B, A @ X, rtol=0, atol=1e-12)
    np.testing.assert_allclose(S, np.abs(A) @ np.abs(X), rtol=1e-13)


def test_canonicalize_sorts_and_inserts_diagonal(oracle_mod):
    m = {"n": 3, "row_ptr": np.array([0, 2, 3, 3], np.int32), "col": np.array([2, 1, 2], np.int32),
         "val": np.array([5.0, 4.0, 1.0])}
    c = oracle_mod.canonicalize(m)
    assert c["row_ptr"].tolist() == [0, 3, 5, 6]
    assert c["col"].tolist() == [0, 1, 2, 1, 2, 2]
    assert c["val"].tolist() == [0.0, 4.0, 5.0, 0.0, 1.0, 0.0]
    with pytest.raises(ValueError):
        oracle_mod.canonicalize({"n": 2, "row_ptr": np.array([0, 0, 1], np.int32),
                                 "col": np.array([0], np.int32), "val": np.array([1.0])})


# ---- closed forms of the synthetic matrices ---------------------------------------------------

def test_anderson_plane_wave_eigenvector(oracle_mod, matgen_mod):
    # W = 0 periodic 7-point hopping -1: A cos(theta.r) = -2 sum_d cos(theta_d) cos(theta.r)
    L = 8
    m = matgen_mod.anderson(L, W=0.0, seed=1)
    assert np.all(m["val"][m["row_ptr"][:-1]] == 0.0)
    x_, y_, z_ = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    th = 2 * np.pi * np.array([1, 2, 3]) / L
    v = np.cos(th[0] * x_ + th[1] * y_ + th[2] * z_).ravel()
    lam = -2.0 * np.cos(th).sum()
    b, _ = oracle_mod.spmv_full(oracle_mod.expand_full(m), v)
    np.testing.assert_allclose(b, lam * v, atol=1e-12)
    np.testing.assert_allclose(oracle_mod.symm_spmv(m, v), lam * v, atol=1e-12)


def test_diagonally_dominant_rows_sum_to_one(oracle_mod, matgen_mod):
    ones = None
    for m in (matgen_mod.stencil3d(9, npt=27, seed=4), matgen_mod.stencil3d(6, 7, 5, npt=7, seed=2),
              matgen_mod.geometric(3000, seed=5), matgen_mod.banded(2000, 60, seed=6)):
        ones = np.ones(m["n"])
        b, _ = oracle_mod.spmv_full(oracle_mod.expand_full(m), ones)
        np.testing.assert_allclose(b, ones, atol=1e-12)


@pytest.mark.parametrize("L", [8, 12, 16])
def test_xxz_uniform_vector_eigenvalue(oracle_mod, matgen_mod, L):
    # periodic chain, Delta = 1: each row sums to J*L/4
    m = matgen_mod.xxz(L)
    n = m["n"]
    assert n == math.comb(L, L // 2)
    b, _ = oracle_mod.spmv_full(oracle_mod.expand_full(m), np.ones(n))
    np.testing.assert_allclose(b, np.full(n, L / 4.0), atol=1e-13)
    # off-diagonal count: L bonds, each antiparallel in 2*C(L-2, L/2-1) states
    offd = len(m["col"]) - n
    assert 2 * offd == L * 2 * math.comb(L - 2, L // 2 - 1)


def test_xxz26_offdiagonals_match_free_fermion_chain_26(matgen_mod):
    # Table "benchmark matrices": FreeFermionChain-26 has 10,400,600 rows and
    # 140,616,112 nonzeros, i.e. exactly the hopping pattern of the periodic
    # L=26 chain; the XXZ matrix adds the (never zero) diagonal.
    m = matgen_mod.xxz(26)
    n = m["n"]
    assert n == 10400600
    assert 2 * (len(m["col"]) - n) == 140616112
    assert np.all(m["val"][m["row_ptr"][:-1]] != 0.0)


@pytest.mark.parametrize("case", ["xxz14", "st27_14", "geo"])
def test_race_threaded_symm_spmv(oracle_mod, matgen_mod, case):
    """The RACE-scheduled multithreaded SymmSpMV (the paper's CPU execution
    model) equals the plain definition within the parity bound, and -- because
    a phase's leaves never share an entry of b -- its result is the same bit
    for bit on 1, 3 and 8 threads."""
    m = {"xxz14": lambda: matgen_mod.xxz(14), "st27_14": lambda: matgen_mod.stencil3d(14, npt=27, seed=2),
         "geo": lambda: matgen_mod.geometric(4000, seed=5, mean_degree=8.0)}[case]()
    sched = oracle_mod.Race(m, 16)
    pm = oracle_mod.permute_upper(m, sched.perm)
    x = matgen_mod.uniform(m["n"], 8, -1.0, 1.0)
    b1 = oracle_mod.symm_spmv_race(pm, sched, x, 1)
    for t in (3, 8):
        assert np.array_equal(oracle_mod.symm_spmv_race(pm, sched, x, t), b1)
    bref, s = oracle_mod.spmv_full(oracle_mod.expand_full(pm), x)
    assert np.all(np.abs(b1 - bref) <= 1e-12 * s + 1e-300)
    # one thread, leaves in schedule order = the serial algorithm on the
    # permuted matrix up to the order of each row's additions
    assert np.allclose(b1, oracle_mod.symm_spmv(pm, x), rtol=0, atol=1e-12 * float(s.max()))


def test_threaded_full_spmv(oracle_mod, matgen_mod):
    m = matgen_mod.anderson(12, W=4.0, seed=3)
    full = oracle_mod.expand_full(m)
    x = matgen_mod.uniform(m["n"], 4, -1.0, 1.0)
    b, _ = oracle_mod.spmv_full(full, x)
    for t in (1, 4):
        assert np.array_equal(oracle_mod.spmv_full_par(full, x, t), b)
    assert oracle_mod.max_threads() >= 1


def test_oracle_error_within_the_recursive_summation_bound(oracle_mod, matgen_mod):
    """The oracle's own FP64 error, against exact rational arithmetic: every
    row of b = A x stays within gamma_m * s_i (m = the row's length,
    gamma_m = m u / (1 - m u), u = 2^-53; Higham, "Accuracy and Stability of
    Numerical Algorithms", Sec. 3.1), far below the 1e-12 * s_i parity bound
    the GPU path is held to."""
    from fractions import Fraction
    m = matgen_mod.stencil3d(7, npt=27, seed=11)
    full = oracle_mod.expand_full(m)
    x = matgen_mod.uniform(m["n"], 12, -1.0, 1.0)
    b, s = oracle_mod.spmv_full(full, x)
    rp, col, val = full["row_ptr"], full["col"], full["val"]
    u = Fraction(1, 2 ** 53)
    worst = 0.0
    for i in range(m["n"]):
        lo, hi = int(rp[i]), int(rp[i + 1])
        exact = sum(Fraction(float(val[j])) * Fraction(float(x[col[j]])) for j in range(lo, hi))
        mlen = hi - lo
        gamma = mlen * u / (1 - mlen * u)
        err = abs(Fraction(float(b[i])) - exact)
        assert err <= gamma * Fraction(float(s[i])) * (1 + 2 * u) + Fraction(1, 2 ** 1074)
        worst = max(worst, float(err / Fraction(float(s[i]))) if s[i] else 0.0)
    assert worst < 1e-15
