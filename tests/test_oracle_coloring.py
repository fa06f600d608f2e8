"""Pins of the oracle's multicolouring schedules (orc_coloring, reading R14):
MC colours rows, ABMC blocks of consecutive rows, first fit in unit order at
graph distance 2.

- closed forms: a path takes colours 0, 1, 2, 0, 1, 2, ...; a star's centre
  and leaves are all pairwise within distance 2 (k + 1 colours); a complete
  graph needs n colours; the 27-point stencil on a lexicographic grid takes
  colour (x mod 3) + 3 (y mod 3) + 9 (z mod 3) (27 colours, 3^3);
- brute force on random matrices (dense distance matrix of the graph): no two
  units of one colour hold rows within distance 2, every row lies in exactly
  one leaf, and every unit's colour is the smallest one not held by an
  earlier unit within distance 2 -- which determines first fit exactly;
- the schedule's layout: units colour by colour, units and rows in order.
"""
import numpy as np
import pytest


def upper(n, edges, diag=2.0):
    rows = [[(i, diag)] for i in range(n)]
    for a, b in edges:
        i, j = min(a, b), max(a, b)
        rows[i].append((j, -1.0))
    rp, col, val = [0], [], []
    for r in rows:
        for c, v in sorted(r):
            col.append(c)
            val.append(v)
        rp.append(len(col))
    return {"n": n, "row_ptr": np.array(rp, np.int32), "col": np.array(col, np.int32), "val": np.array(val)}


def colours(n, sched, bs):
    perm, sp, lo, hi = sched
    col = np.full(n, -1)
    for c in range(len(sp) - 1):
        for q in range(sp[c], sp[c + 1]):
            col[perm[lo[q]:hi[q]]] = c
    return col


def test_path_star_complete(oracle_mod):
    n = 13
    path = upper(n, [(i, i + 1) for i in range(n - 1)])
    assert np.array_equal(colours(n, oracle_mod.coloring(path, 0), 1), np.arange(n) % 3)
    star = upper(9, [(0, i) for i in range(1, 9)])
    assert np.array_equal(colours(9, oracle_mod.coloring(star, 0), 1), np.arange(9))
    k6 = upper(6, [(i, j) for i in range(6) for j in range(i + 1, 6)])
    assert np.array_equal(colours(6, oracle_mod.coloring(k6, 0), 1), np.arange(6))
    # ABMC on the path with blocks of 2: blocks within distance 2 of each other
    # are neighbours in block order, so 2 colours alternate
    assert np.array_equal(colours(n, oracle_mod.coloring(path, 1, 2), 2), (np.arange(n) // 2) % 2)


def test_stencil27_closed_form(oracle_mod, matgen_mod):
    m = matgen_mod.stencil3d(9, npt=27, seed=1)
    idx = np.arange(m["n"])
    x, y, z = idx % 9, (idx // 9) % 9, idx // 81
    assert np.array_equal(colours(m["n"], oracle_mod.coloring(m, 0), 1), (x % 3) + 3 * (y % 3) + 9 * (z % 3))


def distance(m):
    """All-pairs graph distance (BFS), dense; small matrices only."""
    n = m["n"]
    nbr = [[] for _ in range(n)]
    rows = np.repeat(np.arange(n), np.diff(m["row_ptr"]))
    for r, c in zip(rows, m["col"]):
        if r != c:
            nbr[r].append(c)
            nbr[c].append(r)
    D = np.full((n, n), 99, np.int32)
    for s in range(n):
        D[s, s] = 0
        front = [s]
        d = 0
        while front and d < 3:
            d += 1
            nxt = []
            for u in front:
                for v in nbr[u]:
                    if D[s, v] > d:
                        D[s, v] = d
                        nxt.append(v)
            front = nxt
    return D


@pytest.mark.parametrize("which,method,bs", [("geometric", 0, 1), ("geometric", 1, 5), ("band", 0, 1),
                                               ("band", 1, 16), ("xxz", 0, 1), ("xxz", 1, 7)])
def test_first_fit_by_brute_force(oracle_mod, matgen_mod, which, method, bs):
    m = {"geometric": lambda: matgen_mod.geometric(300, seed=8, mean_degree=8.0),
         "band": lambda: matgen_mod.banded(250, 12, seed=2, mean_degree=6.0),
         "xxz": lambda: matgen_mod.xxz(10)}[which]()
    n = m["n"]
    sched = oracle_mod.coloring(m, method, bs)
    perm, sp, lo, hi = sched
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert lo[0] == 0 and hi[-1] == n and np.all(hi[:-1] == lo[1:])
    col = colours(n, sched, bs)
    units = (n + bs - 1) // bs
    D = distance(m)
    near = np.zeros((units, units), bool)  # units with rows within distance 2
    unit_of = np.arange(n) // bs
    ii, jj = np.nonzero(D <= 2)
    near[unit_of[ii], unit_of[jj]] = True
    ucol = np.array([col[u * bs] for u in range(units)])
    for u in range(units):
        assert np.all(col[u * bs:(u + 1) * bs] == ucol[u])
        earlier = np.nonzero(near[u, :u])[0]
        taken = set(ucol[earlier].tolist())
        assert ucol[u] not in taken
        assert all(c in taken for c in range(ucol[u]))  # the smallest free colour
    # layout: units colour by colour, in unit order, rows in order
    want = [r for c in range(len(sp) - 1) for u in range(units) if ucol[u] == c for r in range(u * bs, min(n, (u + 1) * bs))]
    assert np.array_equal(perm, want)
