"""Roofline model of SpMV and SymmSpMV (paper Sec. 3) and GPU traffic figures.

Paper formulas (CPU, with write-allocate on the LHS):
  Eq. "upper_performance":     P = I * b_S
  Eq. "SpMV_intensity":        I_SpMV(alpha)     = 2 / (8 + 4 + 8 alpha + 20 / N_nzr)      flop/byte
  Eq. "SymmSpMV_intensity":    I_SymmSpMV(alpha) = 4 / (8 + 4 + 24 alpha + 4 / N_nzr^symm)
  Eq. "NNZR_symm":             N_nzr^symm = (N_nzr - 1) / 2 + 1
The optimal alpha is 1/N_nzr (SpMV) and 1/N_nzr^symm (SymmSpMV).

GPU algorithmic bytes (no write-allocate; b overwritten, so b is written
once and never has to be read): with v the bytes of a stored value,
  SymmSpMV, k RHS:  (v + 4) nnz_u + 4 (N + 1) + 8 k N (X read) + 8 k N (B written)
  with B read as well (zeroed, accumulated, written back: the paper's count
  at alpha_opt):    (v + 4) nnz_u + 4 N + 24 k N
  full SpMV, k RHS: (v + 4) nnz_f + 4 (N + 1) + 8 k N + 8 k N
Both count every byte the operation must move at least once; flops are
2 nnz_f k for both, so GF/s of the two kernels compare directly.
"""
from __future__ import annotations


def nnzr_symm(nnzr: float) -> float:
    """Eq. NNZR_symm: stored upper nonzeros per row of a symmetric matrix."""
    return (nnzr - 1.0) / 2.0 + 1.0


def i_spmv(alpha: float, nnzr: float) -> float:
    """Eq. SpMV_intensity (flop/byte)."""
    return 2.0 / (8.0 + 4.0 + 8.0 * alpha + 20.0 / nnzr)


def i_symm_spmv(alpha: float, nnzr: float) -> float:
    """Eq. SymmSpMV_intensity (flop/byte); nnzr is the full-matrix N_nzr."""
    return 4.0 / (8.0 + 4.0 + 24.0 * alpha + 4.0 / nnzr_symm(nnzr))


def alpha_from_spmv_bytes(bytes_per_nnz: float, nnzr: float) -> float:
    """Invert the denominator of Eq. SpMV_intensity: measured bytes/nnz -> alpha."""
    return (bytes_per_nnz - 12.0 - 20.0 / nnzr) / 8.0


def perf(intensity: float, bandwidth: float) -> float:
    """Eq. upper_performance: P = I * b_S (units of bandwidth * flop/byte)."""
    return intensity * bandwidth


def symm_bytes(n: int, nnz_u: int, k: int = 1, val_bytes: int = 8) -> int:
    """Minimum bytes of B = A X from upper CRS on a GPU (see module doc)."""
    return (val_bytes + 4) * nnz_u + 4 * (n + 1) + 16 * k * n


def symm_bytes_rmw(n: int, nnz_u: int, k: int = 1, val_bytes: int = 8) -> int:
    """Bytes of B = A X from upper CRS when B is read and written once besides
    X read once: the count of Eq. SymmSpMV_intensity at the optimal alpha
    (24 bytes of vector traffic per row and right-hand side).  The executors
    that zero B and accumulate the transposed update at L2 move this much."""
    return (val_bytes + 4) * nnz_u + 4 * n + 24 * k * n


def full_bytes(n: int, nnz_f: int, k: int = 1, val_bytes: int = 8) -> int:
    """Minimum bytes of B = A X from full CRS on a GPU."""
    return (val_bytes + 4) * nnz_f + 4 * (n + 1) + 16 * k * n


def sweep_bytes(n: int, nnz_f: int, val_bytes: int = 8) -> int:
    """Bytes of one symmetric Gauss-Seidel or Kaczmarz sweep on the full CRS:
    a forward and a backward pass, each reading the matrix, b, and x and
    writing x once."""
    return 2 * ((val_bytes + 4) * nnz_f + 4 * (n + 1) + 24 * n)


def flops(nnz_f: int, k: int = 1) -> int:
    """Useful flops of B = A X (one multiply and one add per full nonzero and column)."""
    return 2 * nnz_f * k
