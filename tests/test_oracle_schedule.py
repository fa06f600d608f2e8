"""Pins of the oracle's RACE schedule.

Against: the numbers the paper prints for its 16x16 walk-through (golden
file), closed-form BFS level sizes, and brute-force distance-2 independence
computed from the sparsity pattern with scipy (A + A^2), which shares nothing
with the oracle.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def stage0_children(r):
    return [r.nodes[c] for c in r.children(0)]


# ---- the paper's worked example ----------------------------------------------------------------

def test_worked_example(oracle_mod, matgen_mod):
    g = golden("paper_worked_example.json")
    m = matgen_mod.paper_stencil2d(16)
    assert m["n"] == g["n_rows"]
    r = oracle_mod.Race(m, g["n_threads"], eps=(g["eps"],) * 8)
    # level sizes 1, 2, 3, ... (weights 1/256*8, 2/256*8, ...)
    d = oracle_mod.bfs_dist(m, m["n"] - 1)
    assert np.bincount(d)[:3].tolist() == g["level_weights_first"]["rows_per_level"]
    ch = stage0_children(r)
    # first pair: seven levels, 28 rows, weight 0.875, one thread
    p0 = ch[0]["nlev"] + ch[1]["nlev"]
    rows0 = ch[0]["size"] + ch[1]["size"]
    assert p0 == g["first_pair"]["levels"] and rows0 == g["first_pair"]["rows"]
    assert rows0 * 8 / 256 == g["first_pair"]["weight"]
    assert ch[0]["nthreads"] == g["first_pair"]["threads"]
    # T0(4)+T0(5): four levels, 54 rows, two threads
    assert ch[4]["nlev"] + ch[5]["nlev"] == g["pair_T0_4_5"]["levels"]
    assert ch[4]["size"] + ch[5]["size"] == g["pair_T0_4_5"]["rows"]
    assert ch[4]["nthreads"] == g["pair_T0_4_5"]["threads"]
    # N_eff(T0(0)) = 15
    assert ch[0]["neff"] == g["T0_0_neff"]["value"]
    # T0(4) = rows 66..90 on threads 2, 3
    t4 = ch[4]
    assert (t4["lo"], t4["hi"] - 1) == (g["T0_4"]["first_row"], g["T0_4"]["last_row"])
    assert list(range(t4["thread_lo"], t4["thread_lo"] + t4["nthreads"])) == g["T0_4"]["threads"]
    # inner four groups recursed into 16 stage-1 groups
    rec = [c for c in ch if c["nchildren"] > 0]
    assert len(rec) == g["recursion"]["recursed_stage0_groups"]
    assert sum(c["nchildren"] for c in rec) == g["recursion"]["stage1_groups"]
    # N_eff(root) = 44, eta = 256/(44*8) = 0.73
    assert r.neff_root() == g["root_neff"]["value"]
    assert round(r.eta, 2) == g["eta"]["printed"]


# ---- level construction against closed forms ---------------------------------------------------

def torus_l1_shell_sizes(L):
    # number of points at L1 distance d on an L^3 torus, from cyclic 1D distances
    one = np.bincount([min(i, L - i) for i in range(L)])
    conv = np.convolve(np.convolve(one, one), one)
    return conv[conv > 0].astype(int).tolist()


@pytest.mark.parametrize("L", [8, 32])
def test_levels_torus(oracle_mod, matgen_mod, L):
    m = matgen_mod.anderson(L, seed=1)
    d = oracle_mod.bfs_dist(m, m["n"] - 1)
    assert np.bincount(d).tolist() == torus_l1_shell_sizes(L)
    assert d.max() + 1 == 3 * (L // 2) + 1


def test_levels_27pt_chebyshev_shells(oracle_mod, matgen_mod):
    n = 12
    m = matgen_mod.stencil3d(n, npt=27)
    d = oracle_mod.bfs_dist(m, m["n"] - 1)
    assert np.bincount(d).tolist() == [(k + 1) ** 3 - k ** 3 for k in range(n)]


def test_stage0_order_is_bfs_order(oracle_mod, matgen_mod):
    m = matgen_mod.anderson(10, seed=3)
    d = oracle_mod.bfs_dist(m, m["n"] - 1)
    r = oracle_mod.Race(m, 8, max_depth=1)
    expect = np.lexsort((np.arange(m["n"]), d))     # by level, then original index
    assert np.array_equal(r.perm, expect)
    assert r.nodes[0]["nsub"] == d.max() + 1


def test_island_level_gap(oracle_mod):
    # two disjoint paths of 5 and 3 vertices: the second island starts two
    # levels after the last level of the first (Sec. 4.4.1)
    edges = [(0, 1), (1, 2), (2, 3), (3, 4), (5, 6), (6, 7)]
    n = 8
    rows = {i: [i] for i in range(n)}
    for a, b in edges:
        rows[min(a, b)].append(max(a, b))
    col = np.concatenate([np.array(sorted(rows[i]), np.int32) for i in range(n)])
    rp = np.concatenate([[0], np.cumsum([len(rows[i]) for i in range(n)])]).astype(np.int32)
    m = {"n": n, "row_ptr": rp, "col": col, "val": np.ones(len(col))}
    r = oracle_mod.Race(m, 1)
    # root = vertex 7: levels 0,1,2 on the 3-path; the 5-path restarts from
    # vertex 4 at level 2+2 = 4 and spans levels 4..8
    assert r.nodes[0]["nsub"] == 9
    assert r.perm.tolist() == [7, 6, 5, 4, 3, 2, 1, 0]


# ---- brute-force distance-2 independence -----------------------------------------------------

def d2_conflicts(pm, stage_ptr, lo, hi):
    """Number of vertex pairs at distance <= 2 that sit in different leaves of one phase."""
    n = pm["n"]
    rows = np.repeat(np.arange(n), np.diff(pm["row_ptr"]))
    A = sp.coo_matrix((np.ones(len(rows)), (rows, pm["col"])), shape=(n, n)).tocsr()
    A = ((A + A.T) > 0).astype(np.int64)
    D2 = ((A + A @ A) > 0).tocoo()
    bad = 0
    for p in range(len(stage_ptr) - 1):
        lab = np.full(n, -1)
        for q in range(stage_ptr[p], stage_ptr[p + 1]):
            lab[lo[q]:hi[q]] = q
        a, b = lab[D2.row], lab[D2.col]
        bad += int(np.count_nonzero((a >= 0) & (b >= 0) & (a != b)))
    return bad


CASES = [
    ("paper16", lambda g: g.paper_stencil2d(16), 8, (0.6,)),
    ("anderson8", lambda g: g.anderson(8, seed=1), 12, (0.8, 0.8, 0.5)),
    ("st27_9", lambda g: g.stencil3d(9, npt=27, seed=4), 6, (0.8, 0.8, 0.5)),
    ("geo", lambda g: g.geometric(2500, seed=5), 16, (0.6, 0.7, 0.5)),
    ("xxz10", lambda g: g.xxz(10), 8, (0.8, 0.8, 0.5)),
    ("band", lambda g: g.banded(1500, 40, seed=2), 20, (0.5,)),
]


@pytest.mark.parametrize("name,mk,nt,eps", CASES)
@pytest.mark.parametrize("max_depth", [-1, 1, 3])
def test_schedule_invariants(oracle_mod, matgen_mod, name, mk, nt, eps, max_depth):
    m = mk(matgen_mod)
    n = m["n"]
    r = oracle_mod.Race(m, nt, eps=eps, max_depth=max_depth)
    assert np.array_equal(np.sort(r.perm), np.arange(n))
    pm = oracle_mod.permute_upper(m, r.perm)
    # every row in exactly one leaf, write sets disjoint inside a phase
    assert oracle_mod.check_phases(pm, r.stage_ptr, r.leaf_lo, r.leaf_hi) == 0
    # distance-2 independence of same-phase leaves (Eq. "corollary_dk")
    assert d2_conflicts(pm, r.stage_ptr, r.leaf_lo, r.leaf_hi) == 0
    for i, nd in enumerate(r.nodes):
        kids = [r.nodes[c] for c in r.children(i)]
        if not kids:
            continue
        assert all(k["nlev"] >= 2 for k in kids)                       # >= k levels per group
        assert sum(k["nthreads"] for k in kids if k["color"] == 0) == nd["nthreads"]
        assert sum(k["nthreads"] for k in kids if k["color"] == 1) == nd["nthreads"]
        assert kids[0]["lo"] == nd["lo"] and kids[-1]["hi"] == nd["hi"]
        assert all(a["hi"] == b["lo"] for a, b in zip(kids, kids[1:]))
        assert [k["color"] for k in kids] == [j % 2 for j in range(len(kids))]
        red = max(k["neff"] for k in kids if k["color"] == 0)
        blue = max(k["neff"] for k in kids if k["color"] == 1)
        assert nd["neff"] == red + blue                                 # Sec. 5 recursion of N_eff
        if max_depth >= 0:
            assert all(k["stage"] < max_depth for k in kids)
    # stage-0 parallelism is bounded by N_l / (2k) pairs
    ch = r.children(0)
    if ch:
        assert len(ch) // 2 <= r.nodes[0]["nsub"] // 4
    assert r.neff_root() >= math.ceil(n / nt)
    assert 0 < r.eta <= 1.0
    assert r.n_phases == r.nodes[0]["phase_count"]


def test_planted_conflicts_are_detected(oracle_mod, matgen_mod):
    m = matgen_mod.anderson(8, seed=1)
    r = oracle_mod.Race(m, 12)
    pm = oracle_mod.permute_upper(m, r.perm)
    sp_, lo, hi = r.stage_ptr.copy(), r.leaf_lo.copy(), r.leaf_hi.copy()
    # merge phase 0 and phase 1 (red and blue groups of one parent touch)
    merged = np.concatenate([[0], sp_[2:]])
    assert oracle_mod.check_phases(pm, merged, lo, hi) == 2
    assert d2_conflicts(pm, merged, lo, hi) > 0
    # drop one leaf: coverage broken
    short_hi = hi.copy()
    short_hi[0] = lo[0] + max(0, (hi[0] - lo[0]) // 2)
    assert oracle_mod.check_phases(pm, sp_, lo, short_hi) == 1


def test_depth_zero_is_one_serial_leaf(oracle_mod, matgen_mod):
    m = matgen_mod.anderson(6, seed=1)
    r = oracle_mod.Race(m, 16, max_depth=0)
    assert r.n_phases == 1 and r.n_leaves == 1
    assert (r.leaf_lo[0], r.leaf_hi[0]) == (0, m["n"])
    assert r.eta == pytest.approx(1.0 / 16)
