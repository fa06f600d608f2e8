"""CPU oracle for the SymmSpMV library — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library (``paper_1907_06487_gb300``)
never does: the oracle is an independent restatement of the paper, written
as plain C (``race_oracle.c``) and wrapped here with ctypes.

Contents (paper: arXiv 1907.06487):
  * ``spmv_full``      Alg. "SpMV using the CRS format" on the symmetric
                       expansion of the upper CRS, with s_i = sum |a_ij||x_j|
  * ``symm_spmv``      Alg. "SymmSpMV", executed serially
  * ``spmv_sampled``   the plain definition for selected rows only
  * ``race``           the RACE schedule (Sec. 4 and 5): levels, pairing by
                       epsilon, load balancing, recursion, tree, eta, phases
  * ``permute_upper``  the symmetric permutation of the upper CRS
  * ``check_phases``   write-set conflict check of a flattened schedule

All functions pinned by tests in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)

DEFAULT_EPS = (0.8, 0.8, 0.5, 0.5, 0.5, 0.5, 0.5, 0.5)


def build_lib(force: bool = False) -> str:
    """Compile race_oracle.c (plain C, -O2, no FP contraction; OpenMP for
    the two multi-threaded baselines when the compiler has it)."""
    src = os.path.join(_HERE, "race_oracle.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, src, "-lm"]
        if subprocess.call(base + ["-fopenmp"], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _get():
    global _lib
    if _lib is not None:
        return _lib
    build_lib()
    L = ctypes.CDLL(_LIB_PATH)
    L.orc_expand_full.restype = ctypes.c_int64
    L.orc_expand_full.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _i64p, _i32p, _f64p]
    L.orc_spmv_full.argtypes = [ctypes.c_int32, _i64p, _i32p, _f64p, _f64p, _f64p, _f64p]
    L.orc_spmm_full.argtypes = [ctypes.c_int32, _i64p, _i32p, _f64p, ctypes.c_int32, _f64p, _f64p, _f64p]
    L.orc_matrix_powers.argtypes = [ctypes.c_int32, _i64p, _i32p, _f64p, ctypes.c_int32, _f64p, _f64p, _f64p,
                                    _f64p]
    L.orc_matrix_powers.restype = None
    L.orc_coloring.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _i32p,
                               _i32p, _i32p]
    L.orc_coloring.restype = ctypes.c_int32
    L.orc_symm_spmv.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
    L.orc_symm_spmv_race.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, ctypes.c_int32, _i32p, _i32p, _i32p,
                                     _f64p, _f64p, ctypes.c_int32]
    L.orc_spmv_full_par.argtypes = [ctypes.c_int32, _i64p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int32]
    L.orc_max_threads.restype = ctypes.c_int32
    L.orc_max_threads.argtypes = []
    L.orc_spmv_sampled.restype = ctypes.c_int
    L.orc_spmv_sampled.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, ctypes.c_int32, _f64p,
                                   ctypes.c_int32, _i32p, _f64p, _f64p]
    L.orc_canonicalize.restype = ctypes.c_int64
    L.orc_canonicalize.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p]
    L.orc_race.restype = ctypes.c_void_p
    L.orc_race.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, _f64p, ctypes.c_int32,
                           ctypes.c_int32, ctypes.c_int32]
    L.orc_race_free.argtypes = [ctypes.c_void_p]
    L.orc_race_info.argtypes = [ctypes.c_void_p, _i32p, _f64p]
    L.orc_race_perm.argtypes = [ctypes.c_void_p, _i32p]
    L.orc_race_phases.argtypes = [ctypes.c_void_p, _i32p, _i32p, _i32p, _i32p]
    L.orc_race_nodes.argtypes = [ctypes.c_void_p, _i32p, _i64p]
    L.orc_race_export.restype = ctypes.c_int64
    L.orc_race_export.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.orc_permute_upper.restype = ctypes.c_int
    L.orc_permute_upper.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p, _i32p, _f64p]
    L.orc_check_phases.restype = ctypes.c_int
    L.orc_check_phases.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, _i32p, _i32p, _i32p]
    L.orc_bfs_dist.restype = ctypes.c_int
    L.orc_bfs_dist.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, _i32p]
    L.orc_pseudo_peripheral.restype = ctypes.c_int32
    L.orc_pseudo_peripheral.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32]
    L.orc_rcm_order.restype = ctypes.c_int32
    L.orc_symm_gs.restype = None
    L.orc_symm_kacz.restype = None
    L.orc_symm_kacz.argtypes = [ctypes.c_int32, _i64p, _i32p, _f64p, ctypes.c_int32, _i32p, _i32p, _i32p, _f64p,
                                _f64p, ctypes.c_int32]
    L.orc_symm_gs.argtypes = [ctypes.c_int32, _i64p, _i32p, _f64p, ctypes.c_int32, _i32p, _i32p, _i32p, _f64p,
                              _f64p, ctypes.c_int32]
    L.orc_rcm_order.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p]
    _lib = L
    return L


def _p(a, t):
    return a.ctypes.data_as(t)


def _mat(m):
    rp = np.ascontiguousarray(m["row_ptr"], dtype=np.int32)
    ci = np.ascontiguousarray(m["col"], dtype=np.int32)
    va = np.ascontiguousarray(m["val"], dtype=np.float64)
    return int(m["n"]), rp, ci, va


def expand_full(m):
    """Full symmetric CRS (int64 row_ptr) from an upper-CRS matrix dict."""
    n, rp, ci, va = _mat(m)
    ndiag = int(np.count_nonzero(ci == np.repeat(np.arange(n, dtype=np.int32), np.diff(rp))))
    nnz_f = 2 * len(ci) - ndiag
    frp = np.zeros(n + 1, np.int64)
    fci = np.zeros(max(nnz_f, 1), np.int32)
    fva = np.zeros(max(nnz_f, 1), np.float64)
    got = _get().orc_expand_full(n, _p(rp, _i32p), _p(ci, _i32p), _p(va, _f64p),
                                 _p(frp, _i64p), _p(fci, _i32p), _p(fva, _f64p))
    assert got == nnz_f
    return {"n": n, "row_ptr": frp, "col": fci[:nnz_f], "val": fva[:nnz_f]}


def spmv_full(full, x):
    """b = A x and s = |A||x| on a full CRS from ``expand_full``."""
    n = full["n"]
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = np.zeros(n); s = np.zeros(n)
    _get().orc_spmv_full(n, _p(full["row_ptr"], _i64p), _p(full["col"], _i32p), _p(full["val"], _f64p),
                         _p(x, _f64p), _p(b, _f64p), _p(s, _f64p))
    return b, s


def spmm_full(full, X):
    """B = A X, S = |A||X| for a row-major n x k block X."""
    n = full["n"]
    X = np.ascontiguousarray(X, dtype=np.float64)
    k = X.shape[1]
    B = np.zeros((n, k)); S = np.zeros((n, k))
    _get().orc_spmm_full(n, _p(full["row_ptr"], _i64p), _p(full["col"], _i32p), _p(full["val"], _f64p),
                         k, _p(X, _f64p), _p(B, _f64p), _p(S, _f64p))
    return B, S


def coloring(m, method, block_rows=1):
    """MC (method 0) or ABMC (method 1, blocks of block_rows rows) schedule of
    an upper-CRS matrix dict: (perm, stage_ptr, leaf_lo, leaf_hi) (R14)."""
    n, rp, ci, va = _mat(m)
    bs = 1 if method == 0 else int(block_rows)
    units = (n + bs - 1) // bs
    perm = np.zeros(max(n, 1), np.int32)
    sp = np.zeros(units + 2, np.int32)
    lo = np.zeros(max(units, 1), np.int32)
    hi = np.zeros(max(units, 1), np.int32)
    nl = np.zeros(1, np.int32)
    ncol = _get().orc_coloring(n, _p(rp, _i32p), _p(ci, _i32p), int(method), bs, _p(perm, _i32p), _p(sp, _i32p),
                               _p(lo, _i32p), _p(hi, _i32p), _p(nl, _i32p))
    return perm[:n], sp[:ncol + 1], lo[:nl[0]], hi[:nl[0]]


def matrix_powers(full, x, p):
    """Y[:, q] = A^(q+1) x and S[:, q] = |A|^(q+1) |x| (n x p arrays) on a full
    CRS from ``expand_full``: the definition applied p times (R13)."""
    n = full["n"]
    x = np.ascontiguousarray(x, dtype=np.float64)
    Y = np.zeros((p, n)); S = np.zeros((p, n)); tmp = np.zeros(n)
    _get().orc_matrix_powers(n, _p(full["row_ptr"], _i64p), _p(full["col"], _i32p), _p(full["val"], _f64p),
                             int(p), _p(x, _f64p), _p(Y, _f64p), _p(S, _f64p), _p(tmp, _f64p))
    return Y.T.copy(), S.T.copy()


def symm_spmv(m, x):
    """Alg. SymmSpMV, serial, b zero-initialised."""
    n, rp, ci, va = _mat(m)
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = np.zeros(n)
    _get().orc_symm_spmv(n, _p(rp, _i32p), _p(ci, _i32p), _p(va, _f64p), _p(x, _f64p), _p(b, _f64p))
    return b


def symm_spmv_race(pm, sched, x, nthreads=0):
    """Alg. SymmSpMV under the RACE schedule `sched` (an oracle ``Race``) on
    CPU threads, phase by phase (the paper's execution model).  `pm` is the
    upper CRS permuted by sched.perm, x in permuted order.  Independent of
    the thread count, bit for bit."""
    n, rp, ci, va = _mat(pm)
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = np.zeros(n)
    _get().orc_symm_spmv_race(n, _p(rp, _i32p), _p(ci, _i32p), _p(va, _f64p), sched.n_phases,
                              _p(sched.stage_ptr, _i32p), _p(sched.leaf_lo, _i32p), _p(sched.leaf_hi, _i32p),
                              _p(x, _f64p), _p(b, _f64p), int(nthreads))
    return b


def spmv_full_par(full, x, nthreads=0):
    """b = A x on a full CRS, rows split over CPU threads."""
    n = full["n"]
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = np.zeros(n)
    _get().orc_spmv_full_par(n, _p(full["row_ptr"], _i64p), _p(full["col"], _i32p), _p(full["val"], _f64p),
                             _p(x, _f64p), _p(b, _f64p), int(nthreads))
    return b


def max_threads() -> int:
    """Threads the oracle's OpenMP loops use by default (1 without OpenMP)."""
    return int(_get().orc_max_threads())


def spmv_sampled(m, X, rows):
    """(b, s) of the plain definition for the given rows (X: n or n x k)."""
    n, rp, ci, va = _mat(m)
    X = np.ascontiguousarray(X, dtype=np.float64)
    k = 1 if X.ndim == 1 else X.shape[1]
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    B = np.zeros((len(rows), k)); S = np.zeros((len(rows), k))
    rc = _get().orc_spmv_sampled(n, _p(rp, _i32p), _p(ci, _i32p), _p(va, _f64p), k, _p(X, _f64p),
                                 len(rows), _p(rows, _i32p), _p(B, _f64p), _p(S, _f64p))
    if rc != 0:
        raise ValueError("bad sample rows")
    if X.ndim == 1:
        return B[:, 0], S[:, 0]
    return B, S


def canonicalize(m):
    """Diagonal-first, sorted upper CRS (explicit 0.0 diagonal when absent)."""
    n, rp, ci, va = _mat(m)
    orp = np.zeros(n + 1, np.int32)
    oci = np.zeros(len(ci) + n, np.int32)
    ova = np.zeros(len(ci) + n, np.float64)
    k = _get().orc_canonicalize(n, _p(rp, _i32p), _p(ci, _i32p), _p(va, _f64p),
                                _p(orp, _i32p), _p(oci, _i32p), _p(ova, _f64p))
    if k < 0:
        raise ValueError("not an upper-triangular CRS")
    return {"n": n, "row_ptr": orp, "col": oci[:k].copy(), "val": ova[:k].copy()}


def bfs_dist(m, root):
    n, rp, ci, _ = _mat(m)
    d = np.zeros(n, np.int32)
    _get().orc_bfs_dist(n, _p(rp, _i32p), _p(ci, _i32p), int(root), _p(d, _i32p))
    return d


def pseudo_peripheral(m, start):
    """George and Liu's pseudo-peripheral vertex reached from `start`."""
    n, rp, ci, _ = _mat(m)
    return int(_get().orc_pseudo_peripheral(n, _p(rp, _i32p), _p(ci, _i32p), int(start)))


def symm_gs(full, stage_ptr, lo, hi, b, x0, sweeps=1):
    """Symmetric Gauss-Seidel sweeps under a flattened schedule (forward over
    the phases, backward in reverse) on a full CRS dict; returns x."""
    n = int(full["n"])
    frp = np.ascontiguousarray(full["row_ptr"], dtype=np.int64)
    fci = np.ascontiguousarray(full["col"], dtype=np.int32)
    fva = np.ascontiguousarray(full["val"], dtype=np.float64)
    sp = np.ascontiguousarray(stage_ptr, dtype=np.int32)
    lo = np.ascontiguousarray(lo, dtype=np.int32)
    hi = np.ascontiguousarray(hi, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    _get().orc_symm_gs(n, _p(frp, _i64p), _p(fci, _i32p), _p(fva, _f64p), len(sp) - 1, _p(sp, _i32p),
                       _p(lo, _i32p), _p(hi, _i32p), _p(b, _f64p), _p(x, _f64p), int(sweeps))
    return x


def symm_kacz(full, stage_ptr, lo, hi, b, x0, sweeps=1):
    """Symmetric Kaczmarz sweeps under a flattened schedule on a full CRS
    dict (same passes as symm_gs; each row projects x onto its hyperplane)."""
    n = int(full["n"])
    frp = np.ascontiguousarray(full["row_ptr"], dtype=np.int64)
    fci = np.ascontiguousarray(full["col"], dtype=np.int32)
    fva = np.ascontiguousarray(full["val"], dtype=np.float64)
    sp = np.ascontiguousarray(stage_ptr, dtype=np.int32)
    lo = np.ascontiguousarray(lo, dtype=np.int32)
    hi = np.ascontiguousarray(hi, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    _get().orc_symm_kacz(n, _p(frp, _i64p), _p(fci, _i32p), _p(fva, _f64p), len(sp) - 1, _p(sp, _i32p),
                         _p(lo, _i32p), _p(hi, _i32p), _p(b, _f64p), _p(x, _f64p), int(sweeps))
    return x


def rcm_order(m):
    """Reverse Cuthill-McKee order, order[new] = old."""
    n, rp, ci, _ = _mat(m)
    out = np.zeros(n, np.int32)
    _get().orc_rcm_order(n, _p(rp, _i32p), _p(ci, _i32p), _p(out, _i32p))
    return out


class Race:
    """The oracle's RACE schedule for one matrix (Sec. 4-5 of the paper)."""

    def __init__(self, m, n_workers, eps=DEFAULT_EPS, max_depth=-1, balance=0, pseudo_peripheral=False, rcm=False,
                 one_level_stage0=False):
        n, rp, ci, _ = _mat(m)
        e = np.zeros(8)
        e[:len(eps)] = eps
        if len(eps) < 8:
            e[len(eps):] = eps[-1]
        self._h = _get().orc_race(n, _p(rp, _i32p), _p(ci, _i32p), int(n_workers), _p(e, _f64p),
                                  int(max_depth), int(balance), int(bool(pseudo_peripheral)) | (2 if rcm else 0)
                                  | (4 if one_level_stage0 else 0))
        if not self._h:
            raise ValueError("oracle race build failed")
        info = np.zeros(6, np.int32)
        eta = ctypes.c_double()
        _get().orc_race_info(self._h, _p(info, _i32p), ctypes.byref(eta))
        self.n, self.n_workers, self.n_nodes, self.n_phases, self.n_leaves, self.depth = (int(v) for v in info)
        self.eta = eta.value
        self.perm = np.zeros(self.n, np.int32)
        _get().orc_race_perm(self._h, _p(self.perm, _i32p))
        self.stage_ptr = np.zeros(self.n_phases + 1, np.int32)
        self.leaf_lo = np.zeros(self.n_leaves, np.int32)
        self.leaf_hi = np.zeros(self.n_leaves, np.int32)
        self.leaf_node = np.zeros(self.n_leaves, np.int32)
        _get().orc_race_phases(self._h, _p(self.stage_ptr, _i32p), _p(self.leaf_lo, _i32p),
                               _p(self.leaf_hi, _i32p), _p(self.leaf_node, _i32p))
        n32 = np.zeros(13 * self.n_nodes, np.int32)
        n64 = np.zeros(2 * self.n_nodes, np.int64)
        _get().orc_race_nodes(self._h, _p(n32, _i32p), _p(n64, _i64p))
        cols = ["parent", "stage", "color", "lo", "hi", "nthreads", "thread_lo", "nlev", "nsub",
                "first_child", "nchildren", "phase_count", "phase_off"]
        n32 = n32.reshape(-1, 13)
        n64 = n64.reshape(-1, 2)
        self.nodes = [dict({c: int(r[j]) for j, c in enumerate(cols)}, size=int(q[0]), neff=int(q[1]))
                      for r, q in zip(n32, n64)]

    def export(self) -> bytes:
        L = _get()
        sz = L.orc_race_export(self._h, None)
        buf = (ctypes.c_uint8 * sz)()
        got = L.orc_race_export(self._h, buf)
        assert got == sz
        return bytes(buf)

    def neff_root(self):
        return self.nodes[0]["neff"]

    def children(self, i):
        nd = self.nodes[i]
        return list(range(nd["first_child"], nd["first_child"] + nd["nchildren"])) if nd["nchildren"] else []

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _get().orc_race_free(h)
            self._h = None


def permute_upper(m, perm):
    """Upper CRS of P A P^T for perm[new] = old."""
    n, rp, ci, va = _mat(m)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    orp = np.zeros(n + 1, np.int32)
    oci = np.zeros(len(ci), np.int32)
    ova = np.zeros(len(ci), np.float64)
    rc = _get().orc_permute_upper(n, _p(rp, _i32p), _p(ci, _i32p), _p(va, _f64p), _p(perm, _i32p),
                                  _p(orp, _i32p), _p(oci, _i32p), _p(ova, _f64p))
    assert rc == 0
    return {"n": n, "row_ptr": orp, "col": oci, "val": ova}


def check_phases(pm, stage_ptr, lo, hi) -> int:
    """0 = conflict-free cover; 1 = a row not covered exactly once; 2 = write conflict in a phase."""
    n, rp, ci, _ = _mat(pm)
    sp = np.ascontiguousarray(stage_ptr, dtype=np.int32)
    lo = np.ascontiguousarray(lo, dtype=np.int32)
    hi = np.ascontiguousarray(hi, dtype=np.int32)
    return int(_get().orc_check_phases(n, _p(rp, _i32p), _p(ci, _i32p), len(sp) - 1, _p(sp, _i32p),
                                       _p(lo, _i32p), _p(hi, _i32p)))
