"""Pins of the oracle's symmetric Gauss-Seidel under a RACE schedule
(orc_symm_gs), the method's other kernel with distance-k dependencies.

A sweep under a schedule is defined as the serial sweep in the schedule's
execution order: forward over the phases (rows of each leaf ascending), then
backward (phases reversed, rows descending).  Checked against what fixes it
independently of the oracle:
- a diagonal matrix is solved exactly by one sweep;
- a forward Gauss-Seidel pass in a row order is the triangular solve
  (D + L) y = b - U x of the matrix permuted into that order (scipy's
  solve_triangular), on the natural order and on RACE execution orders;
- leaves of one phase share no edge, so their order inside the phase does not
  change a single bit; a planted conflict (all leaves in one phase) does;
- on SPD matrices the A-norm of the error falls with every sweep.
"""
import numpy as np
import pytest

scipy_linalg = pytest.importorskip("scipy.linalg")


def dense_full(full):
    n = full["n"]
    A = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(full["row_ptr"]))
    A[rows, full["col"]] = full["val"]
    return A


def forward_pass(A, b, x0, order):
    """Gauss-Seidel pass visiting rows in `order` as a triangular solve."""
    B = A[np.ix_(order, order)]
    L, U = np.tril(B, -1), np.triu(B, 1)
    D = np.diag(np.diag(B))
    y = scipy_linalg.solve_triangular(D + L, b[order] - U @ x0[order], lower=True)
    x = x0.copy()
    x[order] = y
    return x


def execution_orders(sp, lo, hi):
    fwd = [r for ph in range(len(sp) - 1) for q in range(sp[ph], sp[ph + 1]) for r in range(lo[q], hi[q])]
    bwd = [r for ph in reversed(range(len(sp) - 1)) for q in range(sp[ph], sp[ph + 1])
           for r in reversed(range(lo[q], hi[q]))]
    return np.array(fwd), np.array(bwd)


def schedule_full(oracle_mod, m, nt, **kw):
    r = oracle_mod.Race(m, nt, **kw)
    full = oracle_mod.expand_full(oracle_mod.permute_upper(m, r.perm))
    return r, full


def test_diagonal_matrix_one_sweep(oracle_mod):
    n = 40
    d = np.arange(1.0, n + 1)
    m = {"n": n, "row_ptr": np.arange(n + 1, dtype=np.int32), "col": np.arange(n, dtype=np.int32), "val": d}
    r, full = schedule_full(oracle_mod, m, 4)
    b = np.random.default_rng(1).uniform(-1, 1, n)  # in the schedule's order, like x
    d_sched = np.asarray(full["val"])                 # the diagonal, in that order
    assert np.array_equal(np.sort(d_sched), d)
    x = oracle_mod.symm_gs(full, r.stage_ptr, r.leaf_lo, r.leaf_hi, b, np.zeros(n), 1)
    assert np.array_equal(x, b / d_sched)


@pytest.mark.parametrize("name,mk,nt,kw", [
    ("natural", lambda g: g.stencil3d(5, npt=27, seed=3), 1, {"max_depth": 0}),
    ("anderson6", lambda g: g.anderson(6, seed=2), 12, {}),
    ("st27_6_d1", lambda g: g.stencil3d(6, npt=27, seed=5), 16, {"max_depth": 1}),
    ("geo_islands", lambda g: g.geometric(600, seed=3, mean_degree=5.0), 12, {}),
])
def test_sweep_is_the_triangular_solve_in_execution_order(oracle_mod, matgen_mod, name, mk, nt, kw):
    m = mk(matgen_mod)
    r, full = schedule_full(oracle_mod, m, nt, **kw)
    A = dense_full(full)
    n = m["n"]
    rng = np.random.default_rng(7)
    b, x0 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    fwd, bwd = execution_orders(r.stage_ptr, r.leaf_lo, r.leaf_hi)
    want = x0
    for _ in range(2):
        want = forward_pass(A, b, want, fwd)
        want = forward_pass(A, b, want, bwd)
    got = oracle_mod.symm_gs(full, r.stage_ptr, r.leaf_lo, r.leaf_hi, b, x0, 2)
    scale = np.abs(A) @ np.abs(want) + np.abs(b)
    assert np.all(np.abs(got - want) <= 1e-12 * scale)


def reverse_leaves_in_phases(sp, lo, hi):
    lo2, hi2 = lo.copy(), hi.copy()
    for ph in range(len(sp) - 1):
        lo2[sp[ph]:sp[ph + 1]] = lo[sp[ph]:sp[ph + 1]][::-1]
        hi2[sp[ph]:sp[ph + 1]] = hi[sp[ph]:sp[ph + 1]][::-1]
    return lo2, hi2


def edges_between_leaves(full, sp, lo, hi, ph):
    """Edges joining two different leaves of phase ph (brute force)."""
    leaf = np.full(full["n"], -1)
    for q in range(sp[ph], sp[ph + 1]):
        leaf[lo[q]:hi[q]] = q
    rows = np.repeat(np.arange(full["n"]), np.diff(full["row_ptr"]))
    c = full["col"]
    return int(np.count_nonzero((leaf[rows] >= 0) & (leaf[c] >= 0) & (leaf[rows] != leaf[c])))


def test_leaf_order_inside_a_phase_is_irrelevant(oracle_mod, matgen_mod):
    m = matgen_mod.anderson(8, seed=4)
    r, full = schedule_full(oracle_mod, m, 12)
    assert max(np.diff(r.stage_ptr)) > 1
    n = m["n"]
    rng = np.random.default_rng(3)
    b, x0 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    x1 = oracle_mod.symm_gs(full, r.stage_ptr, r.leaf_lo, r.leaf_hi, b, x0, 3)
    lo2, hi2 = reverse_leaves_in_phases(r.stage_ptr, r.leaf_lo, r.leaf_hi)
    x2 = oracle_mod.symm_gs(full, r.stage_ptr, lo2, hi2, b, x0, 3)
    assert np.array_equal(x1, x2)
    assert all(edges_between_leaves(full, r.stage_ptr, r.leaf_lo, r.leaf_hi, ph) == 0
               for ph in range(len(r.stage_ptr) - 1))
    # planted conflict: every leaf in one phase (adjacent leaves now share a
    # phase), so the leaf order matters
    merged = np.array([0, len(r.leaf_lo)], np.int32)
    assert edges_between_leaves(full, merged, r.leaf_lo, r.leaf_hi, 0) > 0
    y1 = oracle_mod.symm_gs(full, merged, r.leaf_lo, r.leaf_hi, b, x0, 1)
    lo3, hi3 = reverse_leaves_in_phases(merged, r.leaf_lo, r.leaf_hi)
    y2 = oracle_mod.symm_gs(full, merged, lo3, hi3, b, x0, 1)
    assert not np.array_equal(y1, y2)


def test_spd_error_falls_in_the_energy_norm(oracle_mod, matgen_mod):
    m = matgen_mod.stencil3d(7, npt=27, seed=8)  # diagonal = row abs sum + 1: SPD
    r, full = schedule_full(oracle_mod, m, 16)
    A = dense_full(full)
    n = m["n"]
    xs = np.random.default_rng(5).uniform(-1, 1, n)
    b = A @ xs
    x = np.zeros(n)
    prev = np.inf
    for _ in range(40):
        x = oracle_mod.symm_gs(full, r.stage_ptr, r.leaf_lo, r.leaf_hi, b, x, 1)
        e = x - xs
        en = float(e @ A @ e)
        assert en < prev
        prev = en
    assert np.linalg.norm(A @ x - b) < 1e-6 * np.linalg.norm(b)


# ------------------------------------------------------------- symmetric Kaczmarz
# A Kaczmarz pass in a row order is a Gauss-Seidel pass on A A^T y = b - A x0
# with x = x0 + A^T y (the rows' projections written in the dual variables),
# a textbook identity independent of the oracle's row loop.

def kaczmarz_pass(A, b, x0, order):
    M = A @ A.T
    y = forward_pass(M, b - A @ x0, np.zeros(len(b)), order)
    return x0 + A.T @ y


@pytest.mark.parametrize("name,mk,nt,kw", [
    ("natural", lambda g: g.stencil3d(5, npt=27, seed=3), 1, {"max_depth": 0}),
    ("anderson6", lambda g: g.anderson(6, seed=2), 12, {}),
    ("st27_6_d1", lambda g: g.stencil3d(6, npt=27, seed=5), 16, {"max_depth": 1}),
])
def test_kaczmarz_is_gauss_seidel_on_the_row_gram_matrix(oracle_mod, matgen_mod, name, mk, nt, kw):
    m = mk(matgen_mod)
    r, full = schedule_full(oracle_mod, m, nt, **kw)
    A = dense_full(full)
    n = m["n"]
    rng = np.random.default_rng(8)
    b, x0 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    fwd, bwd = execution_orders(r.stage_ptr, r.leaf_lo, r.leaf_hi)
    want = kaczmarz_pass(A, b, x0, fwd)
    want = kaczmarz_pass(A, b, want, bwd)
    got = oracle_mod.symm_kacz(full, r.stage_ptr, r.leaf_lo, r.leaf_hi, b, x0, 1)
    assert np.max(np.abs(got - want)) <= 1e-11 * (np.max(np.abs(want)) + 1.0)


def test_kaczmarz_never_moves_away_from_the_solution(oracle_mod, matgen_mod):
    """Each row projection is an orthogonal projection onto a hyperplane that
    contains the solution, so ||x - x*|| cannot grow (any nonsingular A)."""
    m = matgen_mod.anderson(7, seed=3)
    r, full = schedule_full(oracle_mod, m, 16)
    A = dense_full(full)
    n = m["n"]
    xs = np.random.default_rng(2).uniform(-1, 1, n)
    b = A @ xs
    x = np.zeros(n)
    prev = np.linalg.norm(x - xs)
    for _ in range(8):
        x = oracle_mod.symm_kacz(full, r.stage_ptr, r.leaf_lo, r.leaf_hi, b, x, 1)
        cur = np.linalg.norm(x - xs)
        assert cur < prev
        prev = cur


def test_kaczmarz_leaf_order_and_planted_conflict(oracle_mod, matgen_mod):
    m = matgen_mod.anderson(8, seed=4)
    r, full = schedule_full(oracle_mod, m, 12)
    n = m["n"]
    rng = np.random.default_rng(6)
    b, x0 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    x1 = oracle_mod.symm_kacz(full, r.stage_ptr, r.leaf_lo, r.leaf_hi, b, x0, 2)
    lo2, hi2 = reverse_leaves_in_phases(r.stage_ptr, r.leaf_lo, r.leaf_hi)
    assert np.array_equal(x1, oracle_mod.symm_kacz(full, r.stage_ptr, lo2, hi2, b, x0, 2))
    one = np.array([0, len(r.leaf_lo)], np.int32)
    lo3, hi3 = reverse_leaves_in_phases(one, r.leaf_lo, r.leaf_hi)
    assert not np.array_equal(oracle_mod.symm_kacz(full, one, r.leaf_lo, r.leaf_hi, b, x0, 1),
                              oracle_mod.symm_kacz(full, one, lo3, hi3, b, x0, 1))
