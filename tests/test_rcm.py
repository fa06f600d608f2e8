"""CPU tests of the reverse Cuthill-McKee relabelling (RACE_FLAG_RCM), the
ordering the paper applies to all of its inputs before RACE (Sec. 6.1).

The oracle's order is pinned to what the definition and graph theory fix:
- a shuffled path comes out as the path itself, read from one end;
- a level-by-level order has bandwidth at most max_i(|L_i| + |L_{i+1}|) - 1
  over consecutive BFS levels of its start (checked on grids, geometric
  graphs and random graphs with islands);
- Cuthill-McKee's rule, re-derived by brute force from the order alone: every
  vertex's first-reached neighbour is its parent, and the vertices sorted by
  (parent's position, degree, index) reproduce the order; each component
  starts at the pseudo-peripheral vertex reached from its lowest vertex, and
  components come in the order of their lowest vertex.
The library's schedules with the flag equal the oracle's byte for byte.
"""
from collections import deque

import numpy as np
import pytest

import paper_1907_06487_gb300 as R

from test_import_root import adjacency, grid_edges, random_edges, relabel, upper_from_edges


def edges_of(m):
    rp, col = m["row_ptr"], m["col"]
    out = []
    for r in range(m["n"]):
        for t in range(rp[r], rp[r + 1]):
            if col[t] != r:
                out.append((r, int(col[t])))
    return out


def components(n, adj):
    comp = [-1] * n
    k = 0
    for v in range(n):
        if comp[v] >= 0:
            continue
        comp[v] = k
        q = deque([v])
        while q:
            u = q.popleft()
            for w in adj[u]:
                if comp[w] < 0:
                    comp[w] = k
                    q.append(w)
        k += 1
    return comp


def bandwidth(order, edges):
    pos = np.empty(len(order), np.int64)
    pos[np.asarray(order)] = np.arange(len(order))
    return max((abs(int(pos[a]) - int(pos[b])) for a, b in edges if a != b), default=0)


def check_cuthill_mckee(oracle_mod, m, order):
    n = m["n"]
    edges = edges_of(m)
    adj = adjacency(n, edges)
    assert sorted(order) == list(range(n))
    cm = list(order[::-1])
    pos = {v: i for i, v in enumerate(cm)}
    comp = components(n, adj)
    # components in the order of their lowest vertex, each a contiguous block
    # starting at the pseudo-peripheral vertex reached from that lowest vertex
    lowest = {}
    for v in range(n):
        lowest.setdefault(comp[v], v)
    blocks = []
    for i, v in enumerate(cm):
        if i == 0 or comp[v] != comp[cm[i - 1]]:
            blocks.append(i)
    assert len(blocks) == len(lowest)
    assert [lowest[comp[cm[b]]] for b in blocks] == sorted(lowest.values())
    for b in blocks:
        assert cm[b] == oracle_mod.pseudo_peripheral(m, lowest[comp[cm[b]]])
    starts = {cm[b] for b in blocks}
    # breadth first with children by (degree, index): sort key reproduces cm
    key = {}
    for v in cm:
        if v in starts:
            continue
        parent = min(adj[v], key=lambda u: pos[u])
        assert pos[parent] < pos[v]
        key[v] = (comp[v], pos[parent], len(adj[v]), v)
    for b_i, b in enumerate(blocks):
        end = blocks[b_i + 1] if b_i + 1 < len(blocks) else n
        inner = cm[b + 1:end]
        assert inner == sorted(inner, key=lambda v: key[v])


def test_shuffled_path_is_read_end_to_end(oracle_mod):
    n = 57
    p = np.random.default_rng(3).permutation(n)
    edges = [(int(p[i]), int(p[i + 1])) for i in range(n - 1)]
    m = upper_from_edges(n, edges)
    order = list(oracle_mod.rcm_order(m))
    assert order in (list(p), list(p[::-1]))
    assert bandwidth(order, edges) == 1


def level_bound(adj, start):
    d = {start: 0}
    q = deque([start])
    while q:
        u = q.popleft()
        for w in adj[u]:
            if w not in d:
                d[w] = d[u] + 1
                q.append(w)
    sizes = np.bincount(list(d.values()))
    return max((int(sizes[i] + sizes[i + 1]) - 1 for i in range(len(sizes) - 1)), default=0)


GRAPHS = [
    ("grid_8x13", lambda: relabel(104, grid_edges(8, 13), 1), 104),
    ("grid_20x5", lambda: relabel(100, grid_edges(20, 5), 2), 100),
    ("random_islands", lambda: random_edges(400, 420, 7), 400),
    ("random_dense", lambda: random_edges(200, 900, 8), 200),
]


@pytest.mark.parametrize("name,mk,n", GRAPHS, ids=[g[0] for g in GRAPHS])
def test_rcm_definition_and_bandwidth_bound(oracle_mod, name, mk, n):
    edges = mk()
    m = upper_from_edges(n, edges)
    order = oracle_mod.rcm_order(m)
    check_cuthill_mckee(oracle_mod, m, order)
    adj = adjacency(n, edges)
    comp = components(n, adj)
    cm = list(order[::-1])
    bound = 0
    for i, v in enumerate(cm):
        if i == 0 or comp[v] != comp[cm[i - 1]]:
            bound = max(bound, level_bound(adj, v))
    assert bandwidth(order, edges) <= bound


def test_rcm_of_a_shuffled_geometric_graph(oracle_mod, matgen_mod):
    m = matgen_mod.geometric(3000, seed=5)
    p = np.random.default_rng(9).permutation(m["n"])
    shuffled = oracle_mod.permute_upper(m, p)
    order = oracle_mod.rcm_order(shuffled)
    check_cuthill_mckee(oracle_mod, shuffled, order)
    # the relabelling undoes most of the shuffle's damage to the bandwidth
    e = edges_of(shuffled)
    assert bandwidth(order, e) < bandwidth(np.arange(m["n"]), e) / 4


RCM_CASES = [
    ("anderson10", lambda g: g.anderson(10, seed=1), 24, R.PAPER_EPS, -1, 0, False),
    ("geo_islands", lambda g: g.geometric(4000, seed=11), 32, (0.7, 0.6, 0.5), -1, 0, False),
    ("geo_islands_pp", lambda g: g.geometric(4000, seed=11), 32, (0.7, 0.6, 0.5), 1, 0, True),
    ("xxz12_nnz", lambda g: g.xxz(12), 20, R.PAPER_EPS, -1, 1, False),
    ("band_d2", lambda g: g.banded(2500, 90, seed=4), 10, (0.9, 0.8, 0.5), 2, 1, False),
    ("st27_9", lambda g: g.stencil3d(9, npt=27), 16, R.PAPER_EPS, -1, 0, False),
]


@pytest.mark.parametrize("name,mk,nt,eps,md,bal,pp", RCM_CASES, ids=[c[0] for c in RCM_CASES])
def test_rcm_schedule_matches_oracle(oracle_mod, matgen_mod, name, mk, nt, eps, md, bal, pp):
    m = mk(matgen_mod)
    s = R.race_build(m, nt, eps=eps, max_depth=md, balance=bal, host_only=True, rcm=True, pseudo_peripheral=pp)
    o = oracle_mod.Race(m, nt, eps=eps, max_depth=md, balance=bal, rcm=True, pseudo_peripheral=pp)
    assert s.export() == o.export()
    # the permuted matrix is the input permuted by the composed order
    want = oracle_mod.permute_upper(m, s.perm())
    got = s.matrix()
    for k in ("row_ptr", "col", "val"):
        assert np.array_equal(got[k], want[k])


def test_rcm_with_natural_order_is_the_rcm_order(oracle_mod, matgen_mod):
    m = matgen_mod.geometric(2000, seed=3)
    s = R.race_build(m, 8, host_only=True, rcm=True, natural_order=True)
    assert np.array_equal(s.perm(), oracle_mod.rcm_order(m))
    assert s.info()["n_leaves"] == 1


def test_rcm_stage0_root_is_the_first_cm_start(oracle_mod, matgen_mod):
    """After RCM the last row is the first component's Cuthill-McKee start,
    so the default root rule picks it (the paper's setting)."""
    m = matgen_mod.anderson(9, seed=2)
    order = oracle_mod.rcm_order(m)
    s = R.race_build(m, 16, max_depth=1, host_only=True, rcm=True)
    assert s.perm()[0] == order[-1] == oracle_mod.pseudo_peripheral(m, 0)


def test_unknown_flag_bits_are_refused(matgen_mod):
    import ctypes
    m = matgen_mod.anderson(4, seed=1)
    a, keep = R._csr(m, R.RACE_F64)
    p = R.make_params(4, host_only=True)
    p.flags |= 1 << 12
    h = ctypes.c_void_p()
    assert R.lib().race_build(ctypes.byref(a), ctypes.byref(p), None, ctypes.byref(h)) == R.RACE_ERR_INVALID
