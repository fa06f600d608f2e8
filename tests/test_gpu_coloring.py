"""GPU parity of the executors on the MC and ABMC multicolouring schedules
(race_build_coloring) against the oracle: SymmSpMV phase by phase (leaf per
lane group, leaf per block, shared-memory windows) and row-parallel, and the
symmetric Gauss-Seidel sweep in the colouring's execution order, under the
FP64 bound |b_i - b_ref_i| <= 1e-12 sum_j |a_ij||x_j|."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1907_06487_gb300 as R

pytestmark = pytest.mark.gpu

TOL = 1e-12
EXES = [R.RACE_EXEC_LEAF_GROUP, R.RACE_EXEC_LEAF_CTA, R.RACE_EXEC_WINDOW_RACE, R.RACE_EXEC_DF64_RED]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06487_gb300 import build
    build.build()
    return torch.device("cuda:0")


def run(s, x, dev, exe):
    perm = s.perm()
    xd = torch.from_numpy(np.ascontiguousarray(x[perm])).to(dev)
    bd = torch.full_like(xd, np.nan)
    R.symm_spmv_exec(s, exe, xd, bd)
    torch.cuda.synchronize()
    b = np.empty_like(x)
    b[perm] = bd.cpu().numpy()
    return b


@pytest.mark.parametrize("exe", EXES)
@pytest.mark.parametrize("method,bs", [(R.RACE_COLOR_MC, 1), (R.RACE_COLOR_ABMC, 8), (R.RACE_COLOR_ABMC, 64)])
@pytest.mark.parametrize("which", ["st27", "xxz", "geometric"])
def test_symm_spmv_on_colourings(dev, oracle_mod, matgen_mod, which, method, bs, exe):
    m = {"st27": lambda: matgen_mod.stencil3d(14, npt=27, seed=2), "xxz": lambda: matgen_mod.xxz(14),
         "geometric": lambda: matgen_mod.geometric(8000, seed=5, mean_degree=12.0)}[which]()
    s = R.race_build_coloring(m, method, bs, rcm=(which == "geometric"))
    x = matgen_mod.uniform(m["n"], 41, -1.0, 1.0)
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    err = np.abs(run(s, x, dev, exe) - bref)
    assert np.all(err <= TOL * sc + 1e-300), float(np.max(err / (TOL * sc + 1e-300)))


@pytest.mark.parametrize("method,bs", [(R.RACE_COLOR_MC, 1), (R.RACE_COLOR_ABMC, 16)])
def test_gauss_seidel_on_colourings(dev, oracle_mod, matgen_mod, method, bs):
    m = matgen_mod.stencil3d(12, npt=27, seed=7)
    s = R.race_build_coloring(m, method, bs)
    full = oracle_mod.expand_full(s.matrix())
    sp, lo, hi = s.phases()
    rng = np.random.default_rng(2)
    n = m["n"]
    b, x0 = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    want = oracle_mod.symm_gs(full, sp, lo, hi, b, x0, 2)
    bd = torch.from_numpy(b).to(dev)
    xd = torch.from_numpy(x0.copy()).to(dev)
    R.symm_gs(s, bd, xd, 2)
    torch.cuda.synchronize()
    err = np.max(np.abs(xd.cpu().numpy() - want))
    assert err <= 1e-12 * (np.max(np.abs(want)) + np.max(np.abs(x0))), err
