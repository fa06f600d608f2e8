"""GPU parity of the matrix powers (race_matrix_powers, both modes) against the
oracle's plain definition: column q of Y = A^(q+1) x.  The errors of the
successive applications add up through |A|, so power q is held to
(q + 1) * 1e-12 * (|A|^(q+1) |x|)_i per entry.  Cases: stencils, XXZ chains,
band matrices, geometric graphs with islands, natural order, RCM schedules,
p = 1 and p = 64, two calls in a row (the wavefront's flags reset), the
closed-form XXZ eigenvector (every power exact) at full size, and the
refusals."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1907_06487_gb300 as R

pytestmark = pytest.mark.gpu

MODES = [R.RACE_MPK_SWEEPS, R.RACE_MPK_WAVEFRONT]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06487_gb300 import build
    build.build()
    return torch.device("cuda:0")


def powers(s, x, p, mode, dev):
    perm = s.perm()
    n = len(x)
    xd = torch.from_numpy(np.ascontiguousarray(x[perm])).to(dev)
    Yd = torch.full((p * n,), np.nan, dtype=torch.float64, device=dev)
    R.race_matrix_powers(s, p, xd, Yd, mode)
    torch.cuda.synchronize()
    R.race_poll_status(s)
    Yp = Yd.cpu().numpy().reshape(p, n)
    Y = np.empty((n, p))
    Y[perm, :] = Yp.T
    return Y


def check(Y, Yref, S):
    for q in range(Y.shape[1]):
        bound = (q + 1) * 1e-12 * S[:, q] + 1e-300
        err = np.abs(Y[:, q] - Yref[:, q])
        worst = int(np.argmax(err / bound))
        assert np.all(err <= bound), f"power {q + 1}, row {worst}: {err[worst]:.3e} > {bound[worst]:.3e}"


CASES = {
    "st27_15": lambda mg: (mg.stencil3d(15, npt=27, seed=3), {}),
    "xxz14": lambda mg: (mg.xxz(14), {}),
    "band": lambda mg: (mg.banded(7000, 300, seed=4, mean_degree=24.0), {}),
    "geometric_rcm": lambda mg: (mg.geometric(6000, seed=9, mean_degree=6.0), {"rcm": True}),
    "anderson_natural": lambda mg: (mg.anderson(18, seed=5), {"natural_order": True}),
}


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("case", sorted(CASES))
def test_powers_match_oracle(dev, oracle_mod, matgen_mod, case, mode):
    m, kw = CASES[case](matgen_mod)
    s = R.race_build(m, 32, max_depth=1, **kw)
    R.race_set_launch(s, 0, executor=R.RACE_EXEC_DF64_RED, group_lanes=1, rows_per_group=1, blocks_per_sm=0,
                      regs_per_row=4, fp64_quarters=2)
    x = matgen_mod.uniform(m["n"], 23, -1.0, 1.0)
    p = 5
    Yref, S = oracle_mod.matrix_powers(oracle_mod.expand_full(m), x, p)
    check(powers(s, x, p, mode, dev), Yref, S)
    check(powers(s, x, p, mode, dev), Yref, S)  # again: flags and scratch reset


@pytest.mark.parametrize("mode", MODES)
def test_one_power_and_sixty_four(dev, oracle_mod, matgen_mod, mode):
    m = matgen_mod.anderson(9, W=16.5, seed=2)
    s = R.race_build(m, 16)
    x = matgen_mod.uniform(m["n"], 5, -1.0, 1.0) * 0.05  # keeps |A|^64 |x| finite
    for p in (1, 64):
        Yref, S = oracle_mod.matrix_powers(oracle_mod.expand_full(m), x, p)
        check(powers(s, x, p, mode, dev), Yref, S)


@pytest.mark.parametrize("mode", MODES)
def test_fp64_shares_and_x_outside_split_range(dev, oracle_mod, matgen_mod, mode):
    m = matgen_mod.stencil3d(12, npt=27, seed=6)
    s = R.race_build(m, 16)
    x = matgen_mod.uniform(m["n"], 8, -1.0, 1.0)
    x[::37] = 0.0
    x[5::41] = 2.0e20
    p = 3
    Yref, S = oracle_mod.matrix_powers(oracle_mod.expand_full(m), x, p)
    for q64 in (0, 4):
        R.race_set_launch(s, 0, executor=R.RACE_EXEC_DF64_RED, group_lanes=1, rows_per_group=1, blocks_per_sm=0,
                          regs_per_row=4, fp64_quarters=q64)
        check(powers(s, x, p, mode, dev), Yref, S)


def test_xxz26_uniform_vector_exact_at_full_size(dev, matgen_mod):
    """The uniform vector is an eigenvector of the periodic XXZ chain (Delta =
    1) with eigenvalue L/4 = 6.5: every power is exact in binary, on every row
    of the benchmark's matrix and schedule."""
    from paper_1907_06487_gb300 import configs
    m = configs.matrix("xxz26")
    cfg = configs.SCHEDULE["xxz26"]
    s = R.race_build(m, cfg["n_workers"], eps=cfg["eps"], max_depth=cfg["max_depth"], windows=False)
    R.race_set_launch(s, 0, **cfg["launch"])
    n = m["n"]
    x = torch.ones(n, dtype=torch.float64, device=dev)
    p = 3
    for mode in MODES:
        Y = torch.empty(p * n, dtype=torch.float64, device=dev)
        R.race_matrix_powers(s, p, x, Y, mode)
        torch.cuda.synchronize()
        R.race_poll_status(s)
        for q in range(p):
            col = Y[q * n:(q + 1) * n]
            assert bool(torch.all(col == 6.5 ** (q + 1))), (mode, q)
    s.free()


def test_refusals(dev, matgen_mod):
    m = matgen_mod.anderson(6, seed=1)
    s = R.race_build(m, 4)
    n = m["n"]
    x = torch.ones(n, dtype=torch.float64, device=dev)
    Y = torch.empty(4 * n, dtype=torch.float64, device=dev)
    for p, mode, xx in ((0, 0, x), (65, 0, x), (2, 2, x), (2, 1, Y[n:2 * n])):
        with pytest.raises(R.RaceError) as e:
            R.race_matrix_powers(s, p, xx, Y, mode)
        assert e.value.code == R.RACE_ERR_INVALID
    s32 = R.race_build(m, 4, val_type=R.RACE_F32)
    with pytest.raises(R.RaceError) as e:
        R.race_matrix_powers(s32, 2, x, Y, R.RACE_MPK_WAVEFRONT)
    assert e.value.code == R.RACE_ERR_UNSUPPORTED
    R.race_matrix_powers(s32, 2, x, Y, R.RACE_MPK_SWEEPS)
