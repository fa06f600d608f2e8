"""GPU tests of the batch graph and the autotuner (many matrices of uneven
size in one captured CUDA graph; SymmSpMM with k = 4), against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1907_06487_gb300 as R
from paper_1907_06487_gb300 import configs

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06487_gb300 import build
    build.build()
    return torch.device("cuda:0")


def check_rows(B, Bref, S, rows=None):
    err = np.abs(B - Bref)
    bound = TOL * S + 1e-300
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3e}"


def prepare(mats, k, dev, stream, tune=True):
    scheds, Xs, Bs, Xh = [], [], [], []
    for i, m in enumerate(mats):
        s = R.race_build(m, 64, stream=stream)
        n = m["n"]
        X = configs.matgen.uniform(n * k, 300 + i).reshape(n, k)
        perm = s.perm()
        Xd = torch.from_numpy(np.ascontiguousarray(X[perm])).to(dev)
        Bd = torch.empty_like(Xd)
        if tune:
            launch, us = R.race_autotune(s, k, Xd, Bd, reps=2, stream=stream)
            assert launch["executor"] in (R.RACE_EXEC_ROWS_RED, R.RACE_EXEC_PIPE_RED, R.RACE_EXEC_DF64_RED) and us > 0
        scheds.append(s); Xs.append(Xd); Bs.append(Bd); Xh.append(X)
    return scheds, Xs, Bs, Xh


def test_batch_graph_small(dev, oracle_mod):
    k = 4
    mats = configs.batch64(count=8, scale=0.02)
    stream = torch.cuda.Stream(device=dev)
    scheds, Xs, Bs, Xh = prepare(mats, k, dev, stream)
    batch = R.race_batch_create(scheds, k, Xs, Bs, stream)
    for _ in range(2):   # replays overwrite, never accumulate
        batch.launch(stream)
        stream.synchronize()
        for m, s, Bd, X in zip(mats, scheds, Bs, Xh):
            Bref, S = oracle_mod.spmm_full(oracle_mod.expand_full(m), X)
            B = np.empty_like(X)
            B[s.perm()] = Bd.cpu().numpy()
            check_rows(B, Bref, S)
    batch.free()


def test_autotune_keeps_result_correct(dev, oracle_mod, matgen_mod):
    m = matgen_mod.xxz(14)
    s = R.race_build(m, 32)
    x = matgen_mod.uniform(m["n"], 8)
    xd = torch.from_numpy(np.ascontiguousarray(x[s.perm()])).to(dev)
    bd = torch.empty_like(xd)
    launch, us = R.race_autotune(s, 1, xd, bd, reps=3)
    assert R.race_get_launch(s, 0) == launch
    R.symm_spmv(s, xd, bd)
    torch.cuda.synchronize()
    b = np.empty_like(x)
    b[s.perm()] = bd.cpu().numpy()
    bref, sc = oracle_mod.spmv_full(oracle_mod.expand_full(m), x)
    check_rows(b, bref, sc)


def test_batch_rejects_default_stream(dev, matgen_mod):
    m = matgen_mod.anderson(6, seed=1)
    s = R.race_build(m, 4)
    x = torch.zeros(m["n"], dtype=torch.float64, device=dev)
    with pytest.raises(R.RaceError):
        R.race_batch_create([s], 1, [x], [torch.zeros_like(x)], None)


def test_full_size_batch64_sampled(dev, oracle_mod):
    """The 64-matrix batch at full size (k = 4), sampled rows of every matrix."""
    k = 4
    mats = configs.batch64()
    stream = torch.cuda.Stream(device=dev)
    scheds, Xs, Bs, Xh = prepare(mats, k, dev, stream, tune=False)
    batch = R.race_batch_create(scheds, k, Xs, Bs, stream)
    batch.launch(stream)
    stream.synchronize()
    rng = np.random.default_rng(5)
    for m, s, Bd, X in zip(mats, scheds, Bs, Xh):
        n = m["n"]
        rows = np.unique(np.concatenate([[0, n - 1], rng.choice(n, size=min(200, n), replace=False)])).astype(np.int32)
        Bref, S = oracle_mod.spmv_sampled(m, X, rows)
        Bp = Bd.cpu().numpy()
        inv = np.empty(n, np.int64)
        inv[s.perm()] = np.arange(n)
        check_rows(Bp[inv[rows]], Bref, S)
    batch.free()
