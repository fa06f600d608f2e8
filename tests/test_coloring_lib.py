"""The library's MC / ABMC schedules (race_build_coloring) against the
oracle's, byte for byte (permutation, phases, leaves), with and without the
reverse Cuthill-McKee relabelling; their export images import again; the
refusals.  Host only: needs no GPU."""
import numpy as np
import pytest

import paper_1907_06487_gb300 as R
from paper_1907_06487_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return R.lib()


CASES = [("st27_9", lambda mg: mg.stencil3d(9, npt=27, seed=1)), ("xxz12", lambda mg: mg.xxz(12)),
         ("geometric", lambda mg: mg.geometric(4000, seed=6)), ("band", lambda mg: mg.banded(3000, 40, seed=3)),
         ("anderson", lambda mg: mg.anderson(11, seed=2))]


@pytest.mark.parametrize("method,bs", [(R.RACE_COLOR_MC, 1), (R.RACE_COLOR_ABMC, 4), (R.RACE_COLOR_ABMC, 64)])
@pytest.mark.parametrize("name,mk", CASES)
def test_library_matches_oracle(lib, oracle_mod, matgen_mod, name, mk, method, bs):
    m = mk(matgen_mod)
    perm, sp, lo, hi = oracle_mod.coloring(m, method, bs)
    s = R.race_build_coloring(m, method, bs, host_only=True)
    sp2, lo2, hi2 = s.phases()
    assert np.array_equal(s.perm(), perm)
    assert np.array_equal(sp2, sp) and np.array_equal(lo2, lo) and np.array_equal(hi2, hi)
    # the phases are conflict-free on the permuted matrix (the oracle's check)
    pm = oracle_mod.permute_upper(m, perm)
    assert oracle_mod.check_phases(pm, sp, lo, hi) == 0
    t = R.race_import(m, s.export(), host_only=True)
    assert t.export() == s.export()


def test_rcm_relabelling_composes(lib, oracle_mod, matgen_mod):
    m = matgen_mod.geometric(3000, seed=11)
    order = oracle_mod.rcm_order(m)
    mr = oracle_mod.permute_upper(m, order)
    perm, sp, lo, hi = oracle_mod.coloring(mr, R.RACE_COLOR_ABMC, 16)
    s = R.race_build_coloring(m, R.RACE_COLOR_ABMC, 16, host_only=True, rcm=True)
    assert np.array_equal(s.perm(), order[perm])
    sp2, lo2, hi2 = s.phases()
    assert np.array_equal(sp2, sp) and np.array_equal(lo2, lo)


def test_refusals(lib, matgen_mod):
    m = matgen_mod.anderson(5, seed=1)
    for method, bs, nw in ((2, 1, 4), (R.RACE_COLOR_ABMC, 0, 4), (R.RACE_COLOR_ABMC, 4097, 4), (0, 1, 0)):
        with pytest.raises(R.RaceError) as e:
            R.race_build_coloring(m, method, bs, n_workers=nw, host_only=True)
        assert e.value.code == R.RACE_ERR_INVALID
