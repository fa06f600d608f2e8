"""CPU tests of the one-level stage-0 grouping (RACE_FLAG_ONE_LEVEL_STAGE0).

RACE groups at least k = 2 BFS levels so that same-colour groups are
distance-2 independent (Sec. 4.2).  SymmSpMV from half storage needs less:
in level order a row of level j stores only columns of levels j and j + 1
(upper storage; j - 1 and j for lower storage), so it updates b there and
nowhere else, and groups of one level that are one level apart never update
the same entry.  Pinned here by brute force:
- the observation itself on the permuted matrices (every stored upper entry
  goes from level j to level j or j + 1);
- the flagged schedules cover every row once and keep the write sets of the
  leaves of a phase disjoint, with upper and with lower storage, but are not
  distance-2 colourings: an update of every neighbour (the full row's
  pattern, levels j - 1 to j + 1) does conflict, which is why the general
  method needs two levels;
- deeper stages keep two levels per group;
- the library's schedules equal the oracle's byte for byte.
"""
import numpy as np
import pytest

import paper_1907_06487_gb300 as R

from test_oracle_schedule import d2_conflicts

CONNECTED = [
    ("anderson12", lambda g: g.anderson(12, seed=1)),
    ("st27_12", lambda g: g.stencil3d(12, npt=27)),
    ("xxz12", lambda g: g.xxz(12)),
    ("band", lambda g: g.banded(3000, 60, seed=2)),
    ("paper16", lambda g: g.paper_stencil2d(16)),
]


@pytest.mark.parametrize("name,mk", CONNECTED, ids=[c[0] for c in CONNECTED])
def test_upper_entries_reach_only_the_next_level(oracle_mod, matgen_mod, name, mk):
    m = mk(matgen_mod)
    r = oracle_mod.Race(m, 16, max_depth=1)
    pm = oracle_mod.permute_upper(m, r.perm)
    dist = oracle_mod.bfs_dist(pm, 0)  # row 0 of the level order is the root
    assert np.all(dist >= 0) and np.all(np.diff(dist) >= 0)  # levels are contiguous blocks
    rows = np.repeat(np.arange(pm["n"]), np.diff(pm["row_ptr"]))
    step = dist[pm["col"]] - dist[rows]
    assert set(np.unique(step)) <= {0, 1}


def lower_of(pm):
    """Lower-storage CRS of the same matrix: row r lists its columns c <= r."""
    n = pm["n"]
    rows = np.repeat(np.arange(n), np.diff(pm["row_ptr"]))
    order = np.lexsort((rows, pm["col"]))
    r2, c2 = pm["col"][order], rows[order]
    rp = np.concatenate([[0], np.cumsum(np.bincount(r2, minlength=n))]).astype(np.int32)
    return {"n": n, "row_ptr": rp, "col": c2.astype(np.int32), "val": pm["val"][order]}


def full_pattern(oracle_mod, pm):
    """Row r lists every neighbour (the full symmetric row), as int32 CRS."""
    f = oracle_mod.expand_full(pm)
    return {"n": pm["n"], "row_ptr": np.asarray(f["row_ptr"], np.int32), "col": np.asarray(f["col"], np.int32),
            "val": np.asarray(f["val"])}


CASES = [
    ("anderson12", lambda g: g.anderson(12, seed=1), 48),
    ("st27_12", lambda g: g.stencil3d(12, npt=27), 32),
    ("xxz14", lambda g: g.xxz(14), 64),
    ("geo_islands", lambda g: g.geometric(5000, seed=11, mean_degree=6.0), 40),
    ("band", lambda g: g.banded(3000, 60, seed=2), 24),
]


@pytest.mark.parametrize("max_depth", [1, 3, -1])
@pytest.mark.parametrize("name,mk,nt", CASES, ids=[c[0] for c in CASES])
def test_one_level_schedules_are_write_disjoint(oracle_mod, matgen_mod, name, mk, nt, max_depth):
    m = mk(matgen_mod)
    r = oracle_mod.Race(m, nt, max_depth=max_depth, one_level_stage0=True)
    pm = oracle_mod.permute_upper(m, r.perm)
    assert oracle_mod.check_phases(pm, r.stage_ptr, r.leaf_lo, r.leaf_hi) == 0
    assert oracle_mod.check_phases(lower_of(pm), r.stage_ptr, r.leaf_lo, r.leaf_hi) == 0
    for i, nd in enumerate(r.nodes):
        kids = [r.nodes[c] for c in r.children(i)]
        assert all(k["nlev"] >= (1 if i == 0 else 2) for k in kids)
    assert 0 < r.eta <= 1.0


def test_one_level_groups_need_half_storage(oracle_mod, matgen_mod):
    m = matgen_mod.anderson(12, seed=1)
    r = oracle_mod.Race(m, 48, max_depth=1, one_level_stage0=True)
    kids = [r.nodes[c] for c in r.children(0)]
    assert min(k["nlev"] for k in kids) == 1
    pm = oracle_mod.permute_upper(m, r.perm)
    assert oracle_mod.check_phases(pm, r.stage_ptr, r.leaf_lo, r.leaf_hi) == 0
    assert d2_conflicts(pm, r.stage_ptr, r.leaf_lo, r.leaf_hi) > 0
    assert oracle_mod.check_phases(lower_of(pm), r.stage_ptr, r.leaf_lo, r.leaf_hi) == 0
    full = full_pattern(oracle_mod, pm)
    assert oracle_mod.check_phases(full, r.stage_ptr, r.leaf_lo, r.leaf_hi) == 2
    # the two-level schedule is safe for every pattern
    r2 = oracle_mod.Race(m, 48, max_depth=1)
    pm2 = oracle_mod.permute_upper(m, r2.perm)
    for pat in (pm2, lower_of(pm2), full_pattern(oracle_mod, pm2)):
        assert oracle_mod.check_phases(pat, r2.stage_ptr, r2.leaf_lo, r2.leaf_hi) == 0


def test_one_level_doubles_the_stage0_groups(oracle_mod, matgen_mod):
    """Anderson 32^3 from the last vertex: 49 levels; pairs of >= 4 levels
    give at most 12 red/blue pairs, pairs of >= 2 levels up to 24."""
    m = matgen_mod.anderson(32, seed=1)
    two = oracle_mod.Race(m, 64, max_depth=1)
    one = oracle_mod.Race(m, 64, max_depth=1, one_level_stage0=True)
    assert one.nodes[0]["nsub"] == two.nodes[0]["nsub"] == 49
    assert len(two.children(0)) // 2 <= 12
    assert len(one.children(0)) // 2 > 12
    assert one.eta > two.eta


LIB_CASES = [
    ("anderson10", lambda g: g.anderson(10, seed=1), 24, R.PAPER_EPS, -1, 0, {}),
    ("st27_10_d2", lambda g: g.stencil3d(10, npt=27), 16, (0.5, 0.6, 0.5), 2, 0, {}),
    ("geo_islands", lambda g: g.geometric(4000, seed=11), 32, (0.7, 0.6, 0.5), -1, 0, {}),
    ("xxz12_nnz_rcm", lambda g: g.xxz(12), 20, R.PAPER_EPS, -1, 1, {"rcm": True}),
    ("band_pp", lambda g: g.banded(2500, 90, seed=4), 10, (0.9, 0.8, 0.5), 2, 1, {"pseudo_peripheral": True}),
]


@pytest.mark.parametrize("name,mk,nt,eps,md,bal,extra", LIB_CASES, ids=[c[0] for c in LIB_CASES])
def test_one_level_schedule_matches_oracle(oracle_mod, matgen_mod, name, mk, nt, eps, md, bal, extra):
    m = mk(matgen_mod)
    s = R.race_build(m, nt, eps=eps, max_depth=md, balance=bal, host_only=True, one_level_stage0=True, **extra)
    o = oracle_mod.Race(m, nt, eps=eps, max_depth=md, balance=bal, one_level_stage0=True, **extra)
    assert s.export() == o.export()
    # a cached image of it imports (its phases pass the write-set check)
    t = R.race_import(m, s.export(), host_only=True)
    assert t.export() == s.export()
