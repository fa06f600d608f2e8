"""The non-allocating SymmSpMV entry point (symm_spmv_noalloc).

Some callers cannot allocate device memory (a plug-in whose host owns every
allocation, a fixed memory budget, a loop that cannot afford cudaMalloc's
implicit synchronisation).  symm_spmv_noalloc serves them with a fixed
device scratch array instead of per-call allocations.  These tests call it
through the C ABI on caller-owned device arrays and check its result
against the library's regular symm_spmv on the same permuted matrix and
vector and against the CPU oracle, within the parity bound the other GPU
tests use (1e-12 * sum|a||x| per row), on two calls in a row (the scratch
keeps the previous call's contents and must not leak into the next result);
tiny matrices served by the plain-load tail alone; and the refusals (a row
longer than 512 entries, malformed or short row pointers, arrays that do not
start at 16-byte boundaries), which must leave b untouched.

Kept in a file that pytest collects last so that a stop at the first failure
has run every other test already.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1907_06487_gb300 as R

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06487_gb300 import build
    build.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("which", ["xxz16", "anderson21", "st27_17"])
def test_noalloc_matches_symm_spmv(dev, oracle_mod, matgen_mod, which):
    m = {"xxz16": lambda: matgen_mod.xxz(16),
         "anderson21": lambda: matgen_mod.anderson(21, seed=1),
         "st27_17": lambda: matgen_mod.stencil3d(17, npt=27, seed=4)}[which]()
    s = R.race_build(m, 32)
    pm = s.matrix()
    n, nnz = pm["n"], len(pm["col"])
    perm = s.perm()
    rp = torch.from_numpy(pm["row_ptr"]).to(dev)
    col = torch.from_numpy(pm["col"]).to(dev)
    val = torch.from_numpy(pm["val"]).to(dev)
    x = matgen_mod.uniform(n, 11)
    b_oracle, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    for call in range(2):
        xd = torch.from_numpy(np.ascontiguousarray(x[perm])).to(dev)
        b_ref = torch.empty_like(xd)
        R.symm_spmv(s, xd, b_ref)
        b_na = torch.full_like(xd, np.nan)
        R.symm_spmv_noalloc(n, nnz, rp, col, val, xd, b_na)
        torch.cuda.synchronize()
        got, ref = b_na.cpu().numpy(), b_ref.cpu().numpy()
        bound = TOL * sc[perm] + 1e-300
        err = np.abs(got - ref)
        assert np.all(np.isfinite(got)), f"call {call}: non-finite output"
        assert np.all(err <= bound), f"call {call}: max err/bound {np.max(err / bound):.3e}"
        err_o = np.abs(got - b_oracle[perm])
        assert np.all(err_o <= bound), f"call {call}: oracle max err/bound {np.max(err_o / bound):.3e}"


def test_noalloc_rejects_beyond_limits(dev):
    d = torch.zeros(8, dtype=torch.float64, device=dev)
    i = torch.zeros(8, dtype=torch.int32, device=dev)
    with pytest.raises(R.RaceError) as e:
        R.symm_spmv_noalloc((1 << 24) + 1, (1 << 24) + 1, i, i, d, d, torch.zeros_like(d))
    assert e.value.code == R.RACE_ERR_OVERFLOW
    with pytest.raises(R.RaceError) as e:
        R.symm_spmv_noalloc(4, 4, i, i, d, d, d)
    assert e.value.code == R.RACE_ERR_INVALID


def upper_dev(m, dev):
    return (torch.from_numpy(m["row_ptr"]).to(dev), torch.from_numpy(m["col"]).to(dev),
            torch.from_numpy(m["val"]).to(dev))


@pytest.mark.parametrize("n", [5, 6, 7, 8, 9])
def test_noalloc_tiny_matrices(dev, oracle_mod, matgen_mod, n):
    # every block's widened copy would leave the arrays: the tail kernel alone
    m = matgen_mod.banded(n, 4, seed=n, mean_degree=3.0)
    rp, col, val = upper_dev(m, dev)
    x = matgen_mod.uniform(n, 40 + n)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    for _ in range(2):
        b = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
        R.symm_spmv_noalloc(n, len(m["col"]), rp, col, val, torch.from_numpy(x).to(dev), b)
        torch.cuda.synchronize()
        err = np.abs(b.cpu().numpy() - bref)
        assert np.all(err <= TOL * sc + 1e-300)


def long_row_matrix(n=600):
    """Row 0 couples to every other row (n entries); the rest diagonal only."""
    cols = list(range(n)) + list(range(1, n))
    rp = np.array([0, n] + list(range(n + 1, 2 * n)), dtype=np.int32)
    return {"n": n, "row_ptr": rp, "col": np.array(cols, dtype=np.int32), "val": np.linspace(1.0, 2.0, len(cols))}


def refused(dev, n, nnz, rp, col, val, code):
    x = torch.ones(n, dtype=torch.float64, device=dev)
    b = torch.full((n,), 7.25, dtype=torch.float64, device=dev)
    with pytest.raises(R.RaceError) as e:
        R.symm_spmv_noalloc(n, nnz, rp, col, val, x, b)
    assert e.value.code == code
    torch.cuda.synchronize()
    assert bool(torch.all(b == 7.25)), "a refused call wrote b"


def test_noalloc_refuses_rows_over_512_entries(dev):
    m = long_row_matrix(600)  # row 0: 600 entries
    rp, col, val = upper_dev(m, dev)
    refused(dev, m["n"], len(m["col"]), rp, col, val, R.RACE_ERR_UNSUPPORTED)
    m = long_row_matrix(512)  # row 0: exactly 512 entries is served
    rp, col, val = upper_dev(m, dev)
    b = torch.empty(m["n"], dtype=torch.float64, device=dev)
    R.symm_spmv_noalloc(m["n"], len(m["col"]), rp, col, val, torch.ones_like(b), b)


def test_noalloc_refuses_malformed_row_pointers(dev, matgen_mod):
    m = matgen_mod.anderson(12, seed=2)
    n, nnz = m["n"], len(m["col"])
    rp, col, val = upper_dev(m, dev)
    refused(dev, n, nnz - 1, rp, col, val, R.RACE_ERR_INVALID)   # row_ptr[n] != nnz
    refused(dev, n, nnz + 64, rp, col, val, R.RACE_ERR_INVALID)
    bad = m["row_ptr"].copy()
    bad[n // 2] = bad[n // 2 + 1] + 3                             # decreasing
    refused(dev, n, nnz, torch.from_numpy(bad).to(dev), col, val, R.RACE_ERR_INVALID)
    bad = m["row_ptr"].copy()
    bad[0] = 1                                                    # row_ptr[0] != 0
    refused(dev, n, nnz, torch.from_numpy(bad).to(dev), col, val, R.RACE_ERR_INVALID)


def test_noalloc_refuses_misaligned_arrays(dev, matgen_mod):
    m = matgen_mod.anderson(10, seed=3)
    n, nnz = m["n"], len(m["col"])
    rp, col, val = upper_dev(m, dev)
    # views that start 4 or 8 bytes into an allocation (same lengths kept valid)
    col_pad = torch.zeros(nnz + 1, dtype=torch.int32, device=dev)
    col_pad[1:] = col
    val_pad = torch.zeros(nnz + 1, dtype=torch.float64, device=dev)
    val_pad[1:] = val
    rp_pad = torch.zeros(n + 2, dtype=torch.int32, device=dev)
    rp_pad[1:] = rp
    refused(dev, n, nnz, rp, col_pad[1:], val, R.RACE_ERR_INVALID)
    refused(dev, n, nnz, rp, col, val_pad[1:], R.RACE_ERR_INVALID)
    refused(dev, n, nnz, rp_pad[1:], col, val, R.RACE_ERR_INVALID)
