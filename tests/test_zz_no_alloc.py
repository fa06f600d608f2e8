"""The non-allocating SymmSpMV entry point (symm_spmv_noalloc).

Some callers cannot allocate device memory (a plug-in whose host owns every
allocation, a fixed memory budget, a loop that cannot afford cudaMalloc's
implicit synchronisation).  symm_spmv_noalloc serves them with a fixed
device scratch array instead of per-call allocations.  This test calls it
through the C ABI on caller-owned device arrays and checks its result
against the library's regular symm_spmv on the same permuted matrix and
vector, within the parity bound the other GPU tests use (1e-12 * sum|a||x|
per row), on two calls in a row (the scratch keeps the previous call's
contents and must not leak into the next result).

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
    _, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), matgen_mod.uniform(m["n"], 11))
    for call in range(2):
        x = matgen_mod.uniform(n, 11)
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


def test_noalloc_rejects_beyond_limits(dev):
    d = torch.zeros(8, dtype=torch.float64, device=dev)
    i = torch.zeros(8, dtype=torch.int32, device=dev)
    with pytest.raises(R.RaceError) as e:
        R.symm_spmv_noalloc((1 << 24) + 1, (1 << 24) + 1, i, i, d, d, torch.zeros_like(d))
    assert e.value.code == R.RACE_ERR_OVERFLOW
    with pytest.raises(R.RaceError) as e:
        R.symm_spmv_noalloc(4, 4, i, i, d, d, d)
    assert e.value.code == R.RACE_ERR_INVALID
