"""Pins of the oracle's matrix powers (orc_matrix_powers, reading R13):
Y[:, q] = A^(q+1) x and S[:, q] = |A|^(q+1) |x|.

- dense brute force: numpy's matrix_power of the dense symmetric matrix on
  random band, geometric and stencil matrices (catches a power off by one, a
  transposed or half-stored matrix, a wrong magnitude);
- closed forms: the uniform vector is an eigenvector of the periodic XXZ
  Hamiltonian (Delta = 1) with eigenvalue L/4, so every power is exact in
  binary; plane waves are eigenvectors of the disorder-free Anderson model
  with eigenvalue -2 sum_d cos(theta_d);
- a zero vector and p = 1 (one application of the definition).
"""
import numpy as np
import pytest


def dense(m):
    n = m["n"]
    A = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(m["row_ptr"]))
    A[rows, m["col"]] = m["val"]
    A[m["col"], rows] = m["val"]
    return A


@pytest.mark.parametrize("which", ["band", "geometric", "stencil"])
def test_dense_brute_force(oracle_mod, matgen_mod, which):
    m = {"band": lambda: matgen_mod.banded(300, 20, seed=3, mean_degree=8.0),
         "geometric": lambda: matgen_mod.geometric(400, seed=5, mean_degree=10.0),
         "stencil": lambda: matgen_mod.stencil3d(6, npt=27, seed=2)}[which]()
    A = dense(m)
    x = matgen_mod.uniform(m["n"], 17, -1.0, 1.0)
    p = 5
    Y, S = oracle_mod.matrix_powers(oracle_mod.expand_full(m), x, p)
    assert Y.shape == (m["n"], p) and S.shape == (m["n"], p)
    for q in range(p):
        want = np.linalg.matrix_power(A, q + 1) @ x
        want_s = np.linalg.matrix_power(np.abs(A), q + 1) @ np.abs(x)
        assert np.all(np.abs(Y[:, q] - want) <= 1e-13 * want_s + 1e-300)
        assert np.allclose(S[:, q], want_s, rtol=1e-13, atol=0.0)
        assert np.all(np.abs(Y[:, q]) <= S[:, q] * (1 + 1e-13))


@pytest.mark.parametrize("L", [10, 12, 14])
def test_xxz_uniform_vector_is_exact(oracle_mod, matgen_mod, L):
    m = matgen_mod.xxz(L)
    p = 4
    Y, S = oracle_mod.matrix_powers(oracle_mod.expand_full(m), np.ones(m["n"]), p)
    for q in range(p):
        assert np.all(Y[:, q] == (L / 4.0) ** (q + 1))


def test_anderson_plane_wave(oracle_mod, matgen_mod):
    L = 8
    m = matgen_mod.anderson(L, W=0.0, seed=1)
    k = (1, 2, 3)
    th = [2.0 * np.pi * kd / L for kd in k]
    idx = np.arange(L ** 3)
    # lexicographic site index i = x + L (y + L z)
    xs, ys, zs = idx % L, (idx // L) % L, idx // (L * L)
    v = np.cos(th[0] * xs + th[1] * ys + th[2] * zs)
    lam = -2.0 * sum(np.cos(t) for t in th)
    p = 6
    Y, S = oracle_mod.matrix_powers(oracle_mod.expand_full(m), v, p)
    for q in range(p):
        assert np.all(np.abs(Y[:, q] - lam ** (q + 1) * v) <= 1e-12 * S[:, q] + 1e-300)


def test_zero_vector_and_one_power(oracle_mod, matgen_mod):
    m = matgen_mod.anderson(5, seed=2)
    full = oracle_mod.expand_full(m)
    Y, S = oracle_mod.matrix_powers(full, np.zeros(m["n"]), 3)
    assert np.all(Y == 0.0) and np.all(S == 0.0)
    x = matgen_mod.uniform(m["n"], 4)
    Y, S = oracle_mod.matrix_powers(full, x, 1)
    b, s = oracle_mod.spmv_full(full, x)
    assert np.array_equal(Y[:, 0], b) and np.array_equal(S[:, 0], s)
