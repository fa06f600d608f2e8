"""RACE-scheduled symmetric SpMV for GB300 — Python binding of the C ABI.

Argument marshalling only: every step of the path runs in the compiled
library ``_build/librace_gb300.so`` (host schedule builder + sm_103a
kernels).  There is no Python or CPU fallback: if the library is missing the
import of ``lib()`` raises.

Names follow the C ABI in ``include/race.h``:
``race_build``, ``symm_spmv``, ``symm_spmm``, ``spmv_full``, ``race_permute``,
``race_unpermute``, ``race_get_info``, ``race_export``, ``race_import``, ``race_free``.
Device arrays may be torch CUDA tensors (anything with ``data_ptr()``) or raw
integer addresses; streams may be ``torch.cuda.Stream`` objects, raw handles
or None (legacy default stream).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librace_gb300.so")

RACE_OK = 0
RACE_ERR_INVALID = 1
RACE_ERR_OVERFLOW = 2
RACE_ERR_NOMEM = 3
RACE_ERR_CUDA = 4
RACE_ERR_TIMEOUT = 5
RACE_ERR_UNSUPPORTED = 6
RACE_F64 = 0
RACE_F32 = 1
RACE_BAL_ROWS = 0
RACE_BAL_NNZ = 1
RACE_FLAG_HOST_ONLY = 1
RACE_FLAG_NO_WINDOWS = 2
RACE_FLAG_NATURAL_ORDER = 4
RACE_FLAG_PSEUDO_PERIPHERAL = 8
RACE_FLAG_RCM = 16
RACE_FLAG_ONE_LEVEL_STAGE0 = 32

PAPER_EPS = (0.8, 0.8, 0.5, 0.5, 0.5, 0.5, 0.5, 0.5)

# every symbol include/race.h declares
EXPORTED = ("race_default_params", "race_build", "symm_spmv", "symm_spmv_exec", "symm_spmm", "spmv_full",
            "race_prepare_full", "race_permute", "race_unpermute", "race_get_perm", "race_get_matrix",
            "race_get_phases", "race_get_info", "race_export", "race_free", "race_strerror",
            "race_last_error_detail", "race_set_launch", "race_get_launch", "race_poll_status", "race_probe_scatter",
            "symm_spmv_noalloc", "race_batch_create", "race_batch_launch", "race_batch_free", "race_autotune",
            "race_features", "race_mlp_param_count", "race_mlp_act_size", "race_mlp_work_size", "race_mlp_forward",
            "race_mlp_backward", "race_mlp_adam", "race_upload", "race_import", "symm_gs", "symm_kacz",
            "race_probe_wait_timeout", "race_probe_peaks", "race_matrix_powers", "race_probe_reductions",
            "race_build_coloring", "race_probe_barrier_timeout")

RACE_EXEC_LEAF_GROUP = 0
RACE_EXEC_LEAF_CTA = 1
RACE_EXEC_ATOMIC = 2
RACE_EXEC_ROWS_RED = 3
RACE_EXEC_STREAM_RED = 4
RACE_EXEC_PIPE_RED = 5
RACE_EXEC_WINDOW_RED = 6
RACE_EXEC_WINDOW_RACE = 7
RACE_EXEC_DF64_RED = 8
RACE_EXEC_SELL_DF64 = 9
RACE_EXEC_STAGED = 10
RACE_EXEC_PERSIST_GROUP = 11
RACE_EXEC_PERSIST_CTA = 12
RACE_EXEC_PHASE_DF64 = 13


class race_launch(ctypes.Structure):
    _fields_ = [("executor", ctypes.c_int32), ("group_lanes", ctypes.c_int32), ("rows_per_group", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("regs_per_row", ctypes.c_int32),
                ("fp64_quarters", ctypes.c_int32), ("rowsum_fp64_quarters", ctypes.c_int32)]


class RaceError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        detail = ""
        try:
            detail = lib().race_last_error_detail().decode()
        except Exception:  # pragma: no cover - detail is best effort
            pass
        msg = lib().race_strerror(code).decode()
        super().__init__(f"{where}: {msg} (code {code}){': ' + detail if detail else ''}")


class race_csr_upper(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("val_type", ctypes.c_int32)]


class race_params(ctypes.Structure):
    _fields_ = [("dist_k", ctypes.c_int32), ("n_workers", ctypes.c_int32), ("eps", ctypes.c_double * 8),
                ("max_depth", ctypes.c_int32), ("balance", ctypes.c_int32), ("group_lanes", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


class race_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz_upper", ctypes.c_int64), ("n_levels", ctypes.c_int32),
                ("n_phases", ctypes.c_int32), ("n_leaves", ctypes.c_int32), ("n_nodes", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("n_workers", ctypes.c_int32), ("val_type", ctypes.c_int32),
                ("group_lanes", ctypes.c_int32), ("eta", ctypes.c_double), ("neff_root", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """Load the compiled library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} missing: run paper_1907_06487_gb300.build.build() first "
                           "(there is no fallback path)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    L.race_default_params.argtypes = [ctypes.POINTER(race_params), i32]
    L.race_default_params.restype = None
    L.race_build.argtypes = [ctypes.POINTER(race_csr_upper), ctypes.POINTER(race_params), vp, ctypes.POINTER(vp)]
    L.race_build_coloring.argtypes = [ctypes.POINTER(race_csr_upper), i32, i32, i32, ctypes.c_uint32, vp,
                                      ctypes.POINTER(vp)]
    L.race_build_coloring.restype = ctypes.c_int
    for name in ("symm_spmv", "spmv_full"):
        getattr(L, name).argtypes = [vp, vp, vp, vp]
    L.symm_spmm.argtypes = [vp, i32, vp, vp, vp]
    L.symm_spmv_exec.argtypes = [vp, i32, vp, vp, vp]
    L.race_prepare_full.argtypes = [vp, vp]
    L.symm_gs.argtypes = [vp, vp, vp, i32, vp]
    L.symm_kacz.argtypes = [vp, vp, vp, i32, vp]
    L.race_permute.argtypes = [vp, vp, vp, i32, vp]
    L.race_unpermute.argtypes = [vp, vp, vp, i32, vp]
    L.race_get_perm.argtypes = [vp, vp]
    L.race_get_matrix.argtypes = [vp, vp, vp, vp]
    L.race_get_phases.argtypes = [vp, vp, vp, vp]
    L.race_get_info.argtypes = [vp, ctypes.POINTER(race_info)]
    L.race_export.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
    L.race_import.argtypes = [ctypes.POINTER(race_csr_upper), vp, ctypes.c_size_t, ctypes.c_uint32, vp,
                              ctypes.POINTER(vp)]
    L.race_set_launch.argtypes = [vp, i32, ctypes.POINTER(race_launch)]
    L.race_get_launch.argtypes = [vp, i32, ctypes.POINTER(race_launch)]
    L.race_set_launch.restype = ctypes.c_int
    L.race_probe_scatter.argtypes = [vp, i32, vp, vp]
    L.race_probe_scatter.restype = ctypes.c_int
    L.race_poll_status.argtypes = [vp, vp]
    L.race_poll_status.restype = ctypes.c_int
    L.race_probe_peaks.argtypes = [i32, vp, ctypes.c_int64, vp, i32, vp]
    L.race_probe_reductions.argtypes = [i32, vp, ctypes.c_int64, i32, vp, ctypes.c_int64, vp]
    L.race_probe_reductions.restype = ctypes.c_int
    L.race_matrix_powers.argtypes = [vp, i32, vp, vp, i32, vp]
    L.race_matrix_powers.restype = ctypes.c_int
    L.race_probe_peaks.restype = ctypes.c_int
    L.race_probe_wait_timeout.argtypes = [vp, vp, vp, vp]
    L.race_probe_wait_timeout.restype = ctypes.c_int
    L.race_probe_barrier_timeout.argtypes = [vp, vp, vp, vp]
    L.race_probe_barrier_timeout.restype = ctypes.c_int
    L.symm_spmv_noalloc.argtypes = [i32, ctypes.c_int64, vp, vp, vp, vp, vp, vp]
    L.symm_spmv_noalloc.restype = ctypes.c_int
    pvp = ctypes.POINTER(vp)
    L.race_batch_create.argtypes = [pvp, i32, i32, pvp, pvp, vp, pvp]
    L.race_batch_create.restype = ctypes.c_int
    L.race_batch_launch.argtypes = [vp, vp]
    L.race_batch_launch.restype = ctypes.c_int
    L.race_batch_free.argtypes = [vp]
    L.race_batch_free.restype = None
    L.race_autotune.argtypes = [vp, i32, vp, vp, i32, vp, ctypes.POINTER(race_launch), ctypes.POINTER(ctypes.c_float)]
    L.race_autotune.restype = ctypes.c_int
    f32 = ctypes.c_float
    L.race_upload.argtypes = [vp, vp]
    L.race_upload.restype = ctypes.c_int
    L.race_features.argtypes = [ctypes.POINTER(race_csr_upper), vp]
    L.race_features.restype = ctypes.c_int
    L.race_mlp_param_count.argtypes = []
    L.race_mlp_param_count.restype = ctypes.c_int32
    L.race_mlp_act_size.argtypes = [i32]
    L.race_mlp_act_size.restype = ctypes.c_int64
    L.race_mlp_work_size.argtypes = [i32]
    L.race_mlp_work_size.restype = ctypes.c_int64
    L.race_mlp_forward.argtypes = [vp, i32, vp, vp, vp, vp]
    L.race_mlp_forward.restype = ctypes.c_int
    L.race_mlp_backward.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.race_mlp_backward.restype = ctypes.c_int
    L.race_mlp_adam.argtypes = [vp, vp, vp, vp, f32, f32, f32, f32, i32, vp]
    L.race_mlp_adam.restype = ctypes.c_int
    L.race_get_launch.restype = ctypes.c_int
    L.race_free.argtypes = [vp]
    L.race_free.restype = None
    L.race_strerror.argtypes = [ctypes.c_int]
    L.race_strerror.restype = ctypes.c_char_p
    L.race_last_error_detail.argtypes = []
    L.race_last_error_detail.restype = ctypes.c_char_p
    for name in ("race_build", "symm_spmv", "symm_spmv_exec", "symm_spmm", "spmv_full", "race_prepare_full", "race_permute",
                 "race_unpermute", "race_get_perm", "race_get_matrix", "race_get_phases", "race_get_info",
                 "race_export", "race_import", "symm_gs", "symm_kacz"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    raise TypeError(f"cannot take a device pointer of {type(a)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc, where):
    if rc != RACE_OK:
        raise RaceError(rc, where)


def make_params(n_workers, eps=PAPER_EPS, max_depth=-1, balance=RACE_BAL_ROWS, group_lanes=0, host_only=False,
                windows=True, natural_order=False, pseudo_peripheral=False, rcm=False, one_level_stage0=False):
    p = race_params()
    lib().race_default_params(ctypes.byref(p), int(n_workers))
    e = list(eps) + [eps[-1]] * (8 - len(eps))
    for i in range(8):
        p.eps[i] = float(e[i])
    p.max_depth = int(max_depth)
    p.balance = int(balance)
    p.group_lanes = int(group_lanes)
    p.flags = ((RACE_FLAG_HOST_ONLY if host_only else 0) | (0 if windows else RACE_FLAG_NO_WINDOWS)
               | (RACE_FLAG_NATURAL_ORDER if natural_order else 0)
               | (RACE_FLAG_PSEUDO_PERIPHERAL if pseudo_peripheral else 0) | (RACE_FLAG_RCM if rcm else 0)
               | (RACE_FLAG_ONE_LEVEL_STAGE0 if one_level_stage0 else 0))
    return p


class Schedule:
    """Owns a ``race_schedule*``; freed by ``free()`` or garbage collection."""

    def __init__(self, handle, n, k_hint=1):
        self._h = handle
        self.n = n

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("schedule already freed")
        return self._h

    def info(self):
        inf = race_info()
        _check(lib().race_get_info(self.handle, ctypes.byref(inf)), "race_get_info")
        return inf.as_dict()

    def export(self) -> bytes:
        sz = ctypes.c_size_t(0)
        _check(lib().race_export(self.handle, None, ctypes.byref(sz)), "race_export")
        buf = (ctypes.c_uint8 * sz.value)()
        _check(lib().race_export(self.handle, buf, ctypes.byref(sz)), "race_export")
        return bytes(buf)

    def perm(self):
        out = np.zeros(self.n, np.int32)
        _check(lib().race_get_perm(self.handle, out.ctypes.data), "race_get_perm")
        return out

    def matrix(self):
        inf = self.info()
        rp = np.zeros(self.n + 1, np.int32)
        col = np.zeros(inf["nnz_upper"], np.int32)
        val = np.zeros(inf["nnz_upper"], np.float64 if inf["val_type"] == RACE_F64 else np.float32)
        _check(lib().race_get_matrix(self.handle, rp.ctypes.data, col.ctypes.data, val.ctypes.data),
               "race_get_matrix")
        return {"n": self.n, "row_ptr": rp, "col": col, "val": val}

    def phases(self):
        inf = self.info()
        sp = np.zeros(inf["n_phases"] + 1, np.int32)
        lo = np.zeros(inf["n_leaves"], np.int32)
        hi = np.zeros(inf["n_leaves"], np.int32)
        _check(lib().race_get_phases(self.handle, sp.ctypes.data, lo.ctypes.data, hi.ctypes.data), "race_get_phases")
        return sp, lo, hi

    def free(self):
        if getattr(self, "_h", None):
            lib().race_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _csr(m, val_type):
    """race_csr_upper over host arrays; the arrays are returned too and must
    outlive the struct."""
    n = int(m["n"])
    rp = np.ascontiguousarray(m["row_ptr"], dtype=np.int32)
    col = np.ascontiguousarray(m["col"], dtype=np.int32)
    val = np.ascontiguousarray(m["val"], dtype=np.float64 if val_type == RACE_F64 else np.float32)
    a = race_csr_upper(n, int(rp[-1]) if n > 0 else 0, rp.ctypes.data, col.ctypes.data if len(col) else None,
                       val.ctypes.data if len(val) else None, int(val_type))
    return a, (rp, col, val)


def race_build(m, n_workers, eps=PAPER_EPS, max_depth=-1, balance=RACE_BAL_ROWS, group_lanes=0,
               host_only=False, stream=None, val_type=RACE_F64, windows=True, natural_order=False,
               pseudo_peripheral=False, rcm=False, one_level_stage0=False) -> Schedule:
    """race_build on a matrix dict {n, row_ptr, col, val} (host numpy arrays)."""
    a, keep = _csr(m, val_type)
    p = make_params(n_workers, eps, max_depth, balance, group_lanes, host_only, windows, natural_order,
                    pseudo_peripheral, rcm, one_level_stage0)
    h = ctypes.c_void_p()
    _check(lib().race_build(ctypes.byref(a), ctypes.byref(p), _stream(stream), ctypes.byref(h)), "race_build")
    del keep
    return Schedule(h.value, a.n)


RACE_COLOR_MC = 0
RACE_COLOR_ABMC = 1


def race_build_coloring(m, method, block_rows=1, n_workers=152, host_only=False, stream=None, val_type=RACE_F64,
                        windows=True, rcm=False) -> Schedule:
    """race_build_coloring: the MC (rows) or ABMC (blocks of block_rows rows)
    multicolouring schedule of a matrix dict, one phase per colour."""
    a, keep = _csr(m, val_type)
    flags = ((RACE_FLAG_HOST_ONLY if host_only else 0) | (0 if windows else RACE_FLAG_NO_WINDOWS) |
             (RACE_FLAG_RCM if rcm else 0))
    h = ctypes.c_void_p()
    _check(lib().race_build_coloring(ctypes.byref(a), int(method), int(block_rows), int(n_workers), flags,
                                     _stream(stream), ctypes.byref(h)), "race_build_coloring")
    del keep
    return Schedule(h.value, a.n)


def race_import(m, image: bytes, host_only=False, stream=None, val_type=RACE_F64, windows=True) -> Schedule:
    """race_import: the schedule of a race_export image, on the matrix it was built from."""
    a, keep = _csr(m, val_type)
    buf = (ctypes.c_uint8 * len(image)).from_buffer_copy(image) if len(image) else (ctypes.c_uint8 * 1)()
    flags = (RACE_FLAG_HOST_ONLY if host_only else 0) | (0 if windows else RACE_FLAG_NO_WINDOWS)
    h = ctypes.c_void_p()
    _check(lib().race_import(ctypes.byref(a), buf, len(image), flags, _stream(stream), ctypes.byref(h)),
           "race_import")
    del keep
    return Schedule(h.value, a.n)


def symm_spmv(s: Schedule, x, b, stream=None):
    _check(lib().symm_spmv(s.handle, _ptr(x), _ptr(b), _stream(stream)), "symm_spmv")


RACE_MPK_SWEEPS = 0
RACE_MPK_WAVEFRONT = 1


def race_matrix_powers(s: Schedule, p, x, Y, mode=RACE_MPK_WAVEFRONT, stream=None):
    """Y[:, q] = A^(q+1) x (Y: n*p doubles, column q at q*n), permuted order."""
    _check(lib().race_matrix_powers(s.handle, int(p), _ptr(x), _ptr(Y), int(mode), _stream(stream)),
           "race_matrix_powers")


def symm_gs(s: Schedule, b, x, sweeps=1, stream=None):
    """symm_gs: `sweeps` symmetric Gauss-Seidel sweeps on x (in place, permuted order)."""
    _check(lib().symm_gs(s.handle, _ptr(b), _ptr(x), int(sweeps), _stream(stream)), "symm_gs")


def symm_kacz(s: Schedule, b, x, sweeps=1, stream=None):
    """symm_kacz: `sweeps` symmetric Kaczmarz sweeps on x (in place, permuted order)."""
    _check(lib().symm_kacz(s.handle, _ptr(b), _ptr(x), int(sweeps), _stream(stream)), "symm_kacz")


def race_set_launch(s: Schedule, which, executor=0, group_lanes=8, rows_per_group=4, blocks_per_sm=0,
                    regs_per_row=8, fp64_quarters=0, rowsum_fp64_quarters=4):
    """which = 0: symm_spmv, 1: spmv_full."""
    lc = race_launch(int(executor), int(group_lanes), int(rows_per_group), int(blocks_per_sm), int(regs_per_row),
                     int(fp64_quarters), int(rowsum_fp64_quarters))
    _check(lib().race_set_launch(s.handle, int(which), ctypes.byref(lc)), "race_set_launch")


def race_get_launch(s: Schedule, which):
    lc = race_launch()
    _check(lib().race_get_launch(s.handle, int(which), ctypes.byref(lc)), "race_get_launch")
    return {f: getattr(lc, f) for f, _ in lc._fields_}


def race_probe_scatter(s: Schedule, mode, b, stream=None):
    """Diagnostic: mode 0 replays the scatter's reductions, mode 1 its column stream."""
    _check(lib().race_probe_scatter(s.handle, int(mode), _ptr(b), _stream(stream)), "race_probe_scatter")


def race_poll_status(s: Schedule, stream=None):
    _check(lib().race_poll_status(s.handle, _stream(stream)), "race_poll_status")


def race_probe_peaks(what, inp, n, out, iters=1, stream=None):
    """Diagnostic ceilings: what 0 streams n doubles of inp (load-only
    bandwidth), what 1 runs FP64 fused multiply-add chains (iters each)."""
    _check(lib().race_probe_peaks(int(what), _ptr(inp), int(n), _ptr(out), int(iters), _stream(stream)),
           "race_probe_peaks")


def race_probe_reductions(mode, idx, m, max_index, target, n_target, stream=None):
    """Diagnostic: one way of combining scattered contributions (mode 0..4)
    over the target indices idx[0, m)."""
    _check(lib().race_probe_reductions(int(mode), _ptr(idx), int(m), int(max_index), _ptr(target), int(n_target),
                                       _stream(stream)), "race_probe_reductions")


def race_probe_wait_timeout(s: Schedule, x, b, stream=None):
    """Diagnostic: run the staged kernel with waits that give up (b undefined);
    the next race_poll_status then raises RACE_ERR_TIMEOUT once."""
    _check(lib().race_probe_wait_timeout(s.handle, _ptr(x), _ptr(b), _stream(stream)), "race_probe_wait_timeout")


def race_probe_barrier_timeout(s: Schedule, x, b, stream=None):
    """Diagnostic: run the one-launch executor with barriers that expect one
    block too many (b undefined); the next race_poll_status then raises
    RACE_ERR_TIMEOUT once."""
    _check(lib().race_probe_barrier_timeout(s.handle, _ptr(x), _ptr(b), _stream(stream)),
           "race_probe_barrier_timeout")


class Batch:
    """One CUDA graph replaying a SymmSpMV/SymmSpMM per schedule (race_batch_*)."""

    def __init__(self, schedules, k, Xs, Bs, stream):
        n = len(schedules)
        if n < 1 or len(Xs) != n or len(Bs) != n:
            raise ValueError("schedules, Xs and Bs must have the same non-zero length")
        self._keep = (list(schedules), list(Xs), list(Bs))   # device arrays must outlive the graph
        arr = ctypes.c_void_p * n
        h = ctypes.c_void_p()
        _check(lib().race_batch_create(arr(*[s.handle for s in schedules]), n, int(k), arr(*[_ptr(x) for x in Xs]),
                                       arr(*[_ptr(b) for b in Bs]), _stream(stream), ctypes.byref(h)),
               "race_batch_create")
        self._h = h.value

    def launch(self, stream=None):
        _check(lib().race_batch_launch(self._h, _stream(stream)), "race_batch_launch")

    def free(self):
        if getattr(self, "_h", None):
            lib().race_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def race_batch_create(schedules, k, Xs, Bs, stream) -> Batch:
    return Batch(schedules, k, Xs, Bs, stream)


def race_autotune(s: Schedule, k, X, B, reps=5, stream=None):
    """Pick the fastest launch shape for this schedule; returns (launch dict, us per call)."""
    best = race_launch()
    us = ctypes.c_float()
    _check(lib().race_autotune(s.handle, int(k), _ptr(X), _ptr(B), int(reps), _stream(stream), ctypes.byref(best),
                               ctypes.byref(us)), "race_autotune")
    return {f: getattr(best, f) for f, _ in best._fields_}, us.value


def race_upload(s: Schedule, stream=None):
    _check(lib().race_upload(s.handle, _stream(stream)), "race_upload")


def race_features(m, val_type=RACE_F64):
    """16 predictor features of a matrix dict (host numpy arrays)."""
    n = int(m["n"])
    rp = np.ascontiguousarray(m["row_ptr"], dtype=np.int32)
    col = np.ascontiguousarray(m["col"], dtype=np.int32)
    val = np.ascontiguousarray(m["val"], dtype=np.float64)
    a = race_csr_upper(n, int(rp[-1]), rp.ctypes.data, col.ctypes.data if len(col) else None,
                       val.ctypes.data if len(val) else None, RACE_F64)
    out = np.zeros(16, np.float32)
    _check(lib().race_features(ctypes.byref(a), out.ctypes.data), "race_features")
    return out


def race_mlp_forward(params, batch, x, act, y=None, stream=None):
    _check(lib().race_mlp_forward(_ptr(params), int(batch), _ptr(x), _ptr(act), _ptr(y), _stream(stream)),
           "race_mlp_forward")


def race_mlp_backward(params, batch, x, act, target, out_weight, grad, work, loss_terms, stream=None):
    _check(lib().race_mlp_backward(_ptr(params), int(batch), _ptr(x), _ptr(act), _ptr(target), _ptr(out_weight),
                                   _ptr(grad), _ptr(work), _ptr(loss_terms), _stream(stream)), "race_mlp_backward")


def race_mlp_adam(params, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().race_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), float(lr), float(beta1), float(beta2),
                               float(eps), int(step), _stream(stream)), "race_mlp_adam")


def symm_spmv_noalloc(n, nnz, row_ptr, col, val, x, b, stream=None):
    """The non-allocating SymmSpMV: every argument is a caller-owned device array."""
    _check(lib().symm_spmv_noalloc(int(n), int(nnz), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(x), _ptr(b),
                                   _stream(stream)), "symm_spmv_noalloc")


def symm_spmv_exec(s: Schedule, executor, x, b, stream=None):
    _check(lib().symm_spmv_exec(s.handle, int(executor), _ptr(x), _ptr(b), _stream(stream)), "symm_spmv_exec")


def symm_spmm(s: Schedule, k, X, B, stream=None):
    _check(lib().symm_spmm(s.handle, int(k), _ptr(X), _ptr(B), _stream(stream)), "symm_spmm")


def spmv_full(s: Schedule, x, b, stream=None):
    _check(lib().spmv_full(s.handle, _ptr(x), _ptr(b), _stream(stream)), "spmv_full")


def race_prepare_full(s: Schedule, stream=None):
    _check(lib().race_prepare_full(s.handle, _stream(stream)), "race_prepare_full")


def race_permute(s: Schedule, inp, out, k=1, stream=None):
    _check(lib().race_permute(s.handle, _ptr(inp), _ptr(out), int(k), _stream(stream)), "race_permute")


def race_unpermute(s: Schedule, inp, out, k=1, stream=None):
    _check(lib().race_unpermute(s.handle, _ptr(inp), _ptr(out), int(k), _stream(stream)), "race_unpermute")


def race_get_info(s: Schedule):
    return s.info()


def race_export(s: Schedule) -> bytes:
    return s.export()


def race_free(s: Schedule):
    s.free()
