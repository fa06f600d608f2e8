"""Seeded synthetic inputs (matrices in upper-triangle CRS, dense vectors).

Thin ctypes wrapper over ``gen/matgen.c``.  The generated matrices stand in
for the paper's benchmark collection (Table "Details of the benchmark
matrices": Anderson-16.5, Spin-26, HPCG-like stencils); none of the method's
arithmetic lives here, so the CUDA path and the CPU oracle both consume these
inputs.

Every matrix is returned as a dict ``{"n", "row_ptr", "col", "val"}`` with
``row_ptr`` int32 (n+1), ``col`` int32, ``val`` float64, diagonal first in
every row and strictly increasing columns after it.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libmatgen.so")
_lib = None


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.POINTER(ctypes.c_int32)),
                ("col", ctypes.POINTER(ctypes.c_int32)),
                ("val", ctypes.POINTER(ctypes.c_double))]


def build_lib(force: bool = False) -> str:
    """Compile gen/matgen.c into _build/libmatgen.so (host C, no GPU needed)."""
    src = os.path.join(_HERE, "gen", "matgen.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        import subprocess
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _get():
    global _lib
    if _lib is None:
        build_lib()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER(_CSR)
        lib.mg_free.argtypes = [P]
        lib.mg_uniform.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_double)]
        lib.mg_anderson.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, P]
        lib.mg_xxz.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, P]
        lib.mg_stencil3d.argtypes = [ctypes.c_int32] * 3 + [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                            ctypes.c_uint64, P]
        lib.mg_geometric.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, P]
        lib.mg_banded.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, P]
        lib.mg_paper_stencil2d.argtypes = [ctypes.c_int32, ctypes.c_int32, P]
        _lib = lib
    return _lib


def _take(m: _CSR) -> dict:
    n, nnz = m.n, m.nnz
    rp = np.ctypeslib.as_array(m.row_ptr, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(m.col, shape=(nnz,)).copy() if nnz else np.zeros(0, np.int32)
    val = np.ctypeslib.as_array(m.val, shape=(nnz,)).copy() if nnz else np.zeros(0, np.float64)
    _get().mg_free(ctypes.byref(m))
    return {"n": int(n), "row_ptr": rp, "col": col, "val": val}


def _call(fn, *args) -> dict:
    m = _CSR()
    rc = fn(*args, ctypes.byref(m))
    if rc != 0:
        raise ValueError(f"matrix generator failed (rc={rc})")
    return _take(m)


def uniform(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n doubles lo + (hi-lo)*u, u from splitmix64(seed), in index order."""
    out = np.empty(int(n), dtype=np.float64)
    _get().mg_uniform(int(n), int(seed), lo, hi, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def anderson(L: int, W: float = 16.5, seed: int = 1) -> dict:
    """L^3 periodic Anderson model: hopping -1, on-site disorder U[-W/2, W/2)."""
    return _call(_get().mg_anderson, int(L), float(W), int(seed))


def xxz(L: int = 26, J: float = 1.0, Delta: float = 1.0) -> dict:
    """Periodic XXZ chain, Sz=0 sector, basis = ascending L-bit strings with L/2 ones."""
    return _call(_get().mg_xxz, int(L), float(J), float(Delta))


def stencil3d(nx: int, ny: int | None = None, nz: int | None = None, npt: int = 27,
              seed: int = 4, unit_offdiag: bool = False, diag_shift: float = 1.0) -> dict:
    """Nonperiodic 7/27-point stencil; off-diag -U(0,1] (or -1), diag = row abs-sum + shift."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return _call(_get().mg_stencil3d, int(nx), int(ny), int(nz), int(npt), int(unit_offdiag),
                 float(diag_shift), int(seed))


def geometric_radius(npts: int, mean_degree: float = 20.0) -> float:
    """Radius giving the requested nominal mean degree for npts uniform points in the unit cube."""
    return (3.0 * mean_degree / (4.0 * math.pi * npts)) ** (1.0 / 3.0)


def geometric(npts: int, seed: int, mean_degree: float = 20.0, radius: float | None = None) -> dict:
    """Random geometric graph in the unit cube: off-diag -w, w~U(0,1]; diag = sum w + 1."""
    r = geometric_radius(npts, mean_degree) if radius is None else float(radius)
    return _call(_get().mg_geometric, int(npts), r, int(seed))


def banded(n: int, bw: int, seed: int, mean_degree: float = 20.0) -> dict:
    """Random symmetric band matrix of half-bandwidth bw, mean degree ~ mean_degree."""
    p = min(1.0, mean_degree / (2.0 * bw))
    return _call(_get().mg_banded, int(n), int(bw), float(p), int(seed))


def paper_stencil2d(nx: int = 16, ny: int | None = None) -> dict:
    """The walk-through stencil of the paper's Section 4 (5-pt + (+-2,-+2) pair)."""
    ny = nx if ny is None else ny
    return _call(_get().mg_paper_stencil2d, int(nx), int(ny))
