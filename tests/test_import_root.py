"""CPU tests of two parts of the schedule boundary:

- race_import (a schedule rebuilt from a race_export image and its matrix,
  without the construction of Sec. 4): round trips are byte-exact, the
  oracle's images import too, and malformed or mismatched images are refused
  with RACE_ERR_INVALID;
- RACE_FLAG_PSEUDO_PERIPHERAL (stage-0 roots moved to a pseudo-peripheral
  vertex, George and Liu 1979, the start node of the RCM orderings that the
  paper's inputs carry, Sec. 6.1): the oracle's finder is pinned to graphs
  whose peripheral vertices are known (paths, grids, stars) and to the
  finder's stopping rule checked by brute force; the library's schedules
  with the flag equal the oracle's byte for byte.
"""
import struct
from collections import deque

import numpy as np
import pytest

import paper_1907_06487_gb300 as R


def upper_from_edges(n, edges, seed=0):
    """Canonical upper CRS (diagonal first) of the graph with these edges."""
    rng = np.random.default_rng(seed)
    rows = [[(i, 4.0 + rng.random())] for i in range(n)]
    for a, b in edges:
        if a == b:
            continue
        lo, hi = min(a, b), max(a, b)
        rows[lo].append((hi, -rng.random()))
    rp = [0]
    col, val = [], []
    for r in rows:
        first = {}
        for c, v in r[1:]:
            first.setdefault(c, v)  # an edge listed twice is stored once
        r = [r[0]] + sorted(first.items())
        col += [c for c, _ in r]
        val += [v for _, v in r]
        rp.append(len(col))
    return {"n": n, "row_ptr": np.array(rp, np.int32), "col": np.array(col, np.int32), "val": np.array(val)}


def adjacency(n, edges):
    adj = [set() for _ in range(n)]
    for a, b in edges:
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    return adj


def bfs(adj, r):
    d = {r: 0}
    q = deque([r])
    while q:
        u = q.popleft()
        for w in adj[u]:
            if w not in d:
                d[w] = d[u] + 1
                q.append(w)
    return d


def relabel(n, edges, seed):
    p = np.random.default_rng(seed).permutation(n)
    return [(int(p[a]), int(p[b])) for a, b in edges]


def grid_edges(a, b):
    idx = lambda i, j: i * b + j
    e = []
    for i in range(a):
        for j in range(b):
            if i + 1 < a:
                e.append((idx(i, j), idx(i + 1, j)))
            if j + 1 < b:
                e.append((idx(i, j), idx(i, j + 1)))
    return e


def random_edges(n, m, seed):
    rng = np.random.default_rng(seed)
    return [(int(a), int(b)) for a, b in rng.integers(0, n, size=(m, 2))]


# ---------------------------------------------------------------- race_import

IMPORT_CASES = [
    ("anderson8", lambda g: g.anderson(8, seed=1), 16, R.PAPER_EPS, -1, 0),
    ("anderson8_nnz_d2", lambda g: g.anderson(8, seed=1), 24, R.PAPER_EPS, 2, 1),
    ("xxz12", lambda g: g.xxz(12), 20, R.PAPER_EPS, -1, 0),
    ("st27_10_d1", lambda g: g.stencil3d(10, npt=27), 16, R.PAPER_EPS, 1, 0),
    ("geo_islands", lambda g: g.geometric(3000, seed=11), 32, (0.7, 0.6, 0.5), -1, 0),
    ("depth0", lambda g: g.anderson(6, seed=2), 8, R.PAPER_EPS, 0, 0),
]


@pytest.mark.parametrize("name,mk,nt,eps,md,bal", IMPORT_CASES, ids=[c[0] for c in IMPORT_CASES])
def test_import_round_trip(matgen_mod, name, mk, nt, eps, md, bal):
    m = mk(matgen_mod)
    s = R.race_build(m, nt, eps=eps, max_depth=md, balance=bal, host_only=True)
    img = s.export()
    t = R.race_import(m, img, host_only=True)
    assert t.export() == img
    assert t.info() == s.info()
    ms, mt = s.matrix(), t.matrix()
    for k in ("row_ptr", "col", "val"):
        assert np.array_equal(ms[k], mt[k])
    for a, b in zip(s.phases(), t.phases()):
        assert np.array_equal(a, b)


def test_import_of_the_oracles_image(oracle_mod, matgen_mod):
    m = matgen_mod.anderson(8, seed=3)
    img = oracle_mod.Race(m, 12).export()
    t = R.race_import(m, img, host_only=True)
    assert t.export() == img
    assert t.info()["n_levels"] == oracle_mod.Race(m, 12).nodes[0]["nsub"]


def test_import_natural_order_and_fp32(matgen_mod):
    m = matgen_mod.anderson(6, seed=4)
    s = R.race_build(m, 4, natural_order=True, host_only=True)
    t = R.race_import(m, s.export(), host_only=True, val_type=R.RACE_F32)
    assert t.export() == s.export()
    assert t.info()["val_type"] == R.RACE_F32
    assert np.array_equal(t.matrix()["val"], m["val"].astype(np.float32))


def _refused(m, img, fragment=None, flags_host_only=True):
    with pytest.raises(R.RaceError) as e:
        R.race_import(m, img, host_only=flags_host_only)
    assert e.value.code == R.RACE_ERR_INVALID
    if fragment:
        assert fragment in R.lib().race_last_error_detail().decode()


def _header_and_offsets(img, n):
    h = list(struct.unpack_from("<12i", img, 0))
    off_perm = 48 + 72
    off_sp = off_perm + 4 * n
    off_leaf = off_sp + 4 * (h[8] + 1)
    off_tree = off_leaf + 8 * h[9]
    return h, off_perm, off_sp, off_leaf, off_tree


def test_import_refuses_malformed_images(matgen_mod):
    m = matgen_mod.anderson(8, seed=1)
    n = m["n"]
    img = R.race_build(m, 16, host_only=True).export()
    h, off_perm, off_sp, off_leaf, off_tree = _header_and_offsets(img, n)
    assert h[0] == 0x45434152 and h[2] == n and len(img) == off_tree + h[7] * 60
    _refused(m, b"", "header")
    _refused(m, img[:40], "header")
    _refused(m, img[:-1], "size")
    _refused(m, img + b"\0", "size")
    bad = bytearray(img); bad[0] ^= 1
    _refused(m, bytes(bad), "magic")
    bad = bytearray(img); struct.pack_into("<i", bad, 4, 2)
    _refused(m, bytes(bad), "version")
    # perm with a repeated entry
    bad = bytearray(img); struct.pack_into("<i", bad, off_perm, struct.unpack_from("<i", img, off_perm + 4)[0])
    _refused(m, bytes(bad), "permutation")
    # phase offsets that do not end at the leaf count
    bad = bytearray(img); struct.pack_into("<i", bad, off_sp + 4 * h[8], h[9] - 1)
    _refused(m, bytes(bad), "phase")
    # a leaf widened into its neighbour: one row in two leaves
    lo1, hi1 = struct.unpack_from("<2i", img, off_leaf + 8)
    bad = bytearray(img); struct.pack_into("<i", bad, off_leaf + 8, lo1 - 1)
    _refused(m, bytes(bad), "two leaves")
    # an empty leaf
    bad = bytearray(img); struct.pack_into("<i", bad, off_leaf + 12, lo1)
    _refused(m, bytes(bad), "leaf")
    # the root claims more children than there are nodes
    bad = bytearray(img); struct.pack_into("<i", bad, off_tree + 8 * 4, h[7])
    _refused(m, bytes(bad), "tree")
    # flags other than host-only and no-windows
    a, keep = R._csr(m, R.RACE_F64)
    import ctypes
    buf = (ctypes.c_uint8 * len(img)).from_buffer_copy(img)
    hnd = ctypes.c_void_p()
    rc = R.lib().race_import(ctypes.byref(a), buf, len(img), R.RACE_FLAG_NATURAL_ORDER, None, ctypes.byref(hnd))
    assert rc == R.RACE_ERR_INVALID and not hnd.value


def test_import_refuses_an_image_of_another_matrix(matgen_mod):
    m = matgen_mod.anderson(8, seed=1)
    img = R.race_build(m, 16, host_only=True).export()
    _refused(matgen_mod.anderson(7, seed=1), img, "rows")
    # same size, denser graph: the image's phases are not a distance-2
    # colouring of it
    n = m["n"]
    band = upper_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, min(n, i + 40))])
    _refused(band, img, "distance-2")
    # same graph, other values: accepted, and the values are the new ones
    m2 = dict(m, val=m["val"] * 2.0)
    t = R.race_import(m2, img, host_only=True)
    assert np.array_equal(t.matrix()["val"], R.race_build(m2, 16, host_only=True).matrix()["val"])


# ------------------------------------------------------ pseudo-peripheral root

def ecc(adj, r):
    return max(bfs(adj, r).values())


def test_pseudo_peripheral_path(oracle_mod):
    n = 40
    edges = relabel(n, [(i, i + 1) for i in range(n - 1)], seed=1)
    m = upper_from_edges(n, edges)
    adj = adjacency(n, edges)
    for start in (0, 7, n // 2, n - 1):
        r = oracle_mod.pseudo_peripheral(m, start)
        assert len(adj[r]) == 1 and ecc(adj, r) == n - 1  # an end of the path


@pytest.mark.parametrize("a,b", [(7, 11), (9, 9), (1, 6), (4, 15)])
def test_pseudo_peripheral_grid_is_a_corner(oracle_mod, a, b):
    n = a * b
    edges = relabel(n, grid_edges(a, b), seed=a * 100 + b)
    m = upper_from_edges(n, edges)
    adj = adjacency(n, edges)
    diameter = max(ecc(adj, v) for v in range(n))
    assert diameter == a + b - 2
    for start in (0, n // 3, n - 1):
        r = oracle_mod.pseudo_peripheral(m, start)
        assert ecc(adj, r) == diameter
        assert len(adj[r]) == (1 if min(a, b) == 1 else 2)  # a corner


def test_pseudo_peripheral_star_and_isolated(oracle_mod):
    n = 12
    edges = [(0, i) for i in range(1, n - 1)]  # vertex n-1 is isolated
    m = upper_from_edges(n, edges)
    assert oracle_mod.pseudo_peripheral(m, n - 1) == n - 1
    r = oracle_mod.pseudo_peripheral(m, 0)
    assert r == 1  # every leaf is farthest from the centre, all of degree 1: lowest index
    assert oracle_mod.pseudo_peripheral(m, 5) == 5  # a leaf: its farthest set holds no better vertex


@pytest.mark.parametrize("seed", range(6))
def test_pseudo_peripheral_stopping_rule(oracle_mod, seed):
    """On random graphs with islands: the result lies in the start's
    component, is at least as eccentric as the start, and the rule's next
    candidate (minimum degree, lowest index, among its farthest vertices)
    is not more eccentric."""
    n = 300
    edges = random_edges(n, 330, seed)
    m = upper_from_edges(n, edges)
    adj = adjacency(n, edges)
    for start in (n - 1, 0, 123):
        r = oracle_mod.pseudo_peripheral(m, start)
        dr = bfs(adj, r)
        assert start in dr
        e = max(dr.values())
        assert e >= ecc(adj, start)
        far = [v for v, d in dr.items() if d == e]
        x = min(far, key=lambda v: (len(adj[v]), v))
        assert ecc(adj, x) <= e


def test_library_stage0_root_is_the_oracles(oracle_mod, matgen_mod):
    """With max_depth 1 the schedule's first row is the stage-0 root."""
    for m in (matgen_mod.anderson(9, seed=1), matgen_mod.xxz(12), matgen_mod.stencil3d(9, npt=27)):
        n = m["n"]
        s = R.race_build(m, 16, max_depth=1, host_only=True, pseudo_peripheral=True)
        assert s.perm()[0] == oracle_mod.pseudo_peripheral(m, n - 1)
        assert R.race_build(m, 16, max_depth=1, host_only=True).perm()[0] == n - 1


PP_CASES = [
    ("anderson10", lambda g: g.anderson(10, seed=1), 24, R.PAPER_EPS, -1, 0),
    ("st27_10", lambda g: g.stencil3d(10, npt=27), 16, (0.5, 0.6, 0.5), 3, 0),
    ("geo_islands", lambda g: g.geometric(4000, seed=11), 32, (0.7, 0.6, 0.5), -1, 0),
    ("xxz12_nnz", lambda g: g.xxz(12), 20, R.PAPER_EPS, -1, 1),
    ("band", lambda g: g.banded(2500, 90, seed=4), 10, (0.9, 0.8, 0.5), 2, 1),
]


@pytest.mark.parametrize("name,mk,nt,eps,md,bal", PP_CASES, ids=[c[0] for c in PP_CASES])
def test_pseudo_peripheral_schedule_matches_oracle(oracle_mod, matgen_mod, name, mk, nt, eps, md, bal):
    m = mk(matgen_mod)
    s = R.race_build(m, nt, eps=eps, max_depth=md, balance=bal, host_only=True, pseudo_peripheral=True)
    o = oracle_mod.Race(m, nt, eps=eps, max_depth=md, balance=bal, pseudo_peripheral=True)
    assert s.export() == o.export()


def test_pseudo_peripheral_on_a_shuffled_path_restores_the_order(oracle_mod):
    """A path whose vertices are shuffled: from the default root (the last
    vertex, somewhere inside the path) the levels fold the path in two; from
    the pseudo-peripheral root every level holds one vertex and the
    permutation walks the path end to end."""
    n = 64
    p = np.random.default_rng(5).permutation(n)
    edges = [(int(p[i]), int(p[i + 1])) for i in range(n - 1)]
    m = upper_from_edges(n, edges)
    s = R.race_build(m, 4, max_depth=1, host_only=True, pseudo_peripheral=True)
    order = s.perm()
    assert sorted(order) == list(range(n))
    assert list(order) in (list(p), list(p[::-1]))
    assert s.info()["n_levels"] == n
    assert R.race_build(m, 4, max_depth=1, host_only=True).info()["n_levels"] < n


def test_pseudo_peripheral_with_natural_order_is_refused(matgen_mod):
    with pytest.raises(R.RaceError) as e:
        R.race_build(matgen_mod.anderson(4, seed=1), 4, host_only=True, natural_order=True, pseudo_peripheral=True)
    assert e.value.code == R.RACE_ERR_INVALID
