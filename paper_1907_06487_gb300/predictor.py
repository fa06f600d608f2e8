"""Learned RACE-parameter predictor.

The paper fixes the schedule parameters by a parameter study (Sec. 5.1:
eps_{0,1} = 0.8, eps_{s>1} = 0.5, recursion as deep as the epsilon rule
goes).  Here a small perceptron (16 -> 64 -> 64 -> 3, hand-written CUDA
forward/backward/Adam kernels behind the C ABI) predicts (eps_0, eps_1,
depth) from 16 matrix features (race_features), trained on timings the
method itself produces: for every training matrix the grid
eps_0, eps_1 in {0.5, 0.6, 0.7, 0.8, 0.9} x depth in {1, 2, 3, 4, unlimited}
(eps_s = 0.5 for s > 1) is swept, each point timed on the GPU with the
schedule-bound executor (RACE_EXEC_LEAF_GROUP: one RACE leaf per lane group,
plain stores, one launch per phase), and the fastest point is the label.
The exhaustive sweep stays both the fallback and the judge of the
predictor's regret.

Usage (GPU):  python -m paper_1907_06487_gb300.predictor sweep   (writes data/predictor_sweep.npz)
              python -m paper_1907_06487_gb300.predictor train   (writes data/predictor.f32)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

from . import RACE_EXEC_LEAF_GROUP, lib, matgen, race_build, race_features, symm_spmv_exec
from . import race_mlp_adam, race_mlp_backward, race_mlp_forward

GRID_EPS = (0.5, 0.6, 0.7, 0.8, 0.9)
GRID_DEPTH = (1, 2, 3, 4, -1)
GRID = [(e0, e1, d) for e0 in GRID_EPS for e1 in GRID_EPS for d in GRID_DEPTH]
PAPER_POINT = (0.8, 0.8, -1)
SWEEP_WORKERS = 128
HERE = os.path.dirname(os.path.abspath(__file__))
DATA = os.path.join(HERE, "data")


def point_index(e0, e1, d):
    return GRID.index((e0, e1, d))


def encode(e0, e1, d):
    """Target in [0,1]^3 for a grid point."""
    return np.array([(e0 - 0.5) / 0.4, (e1 - 0.5) / 0.4, GRID_DEPTH.index(d) / 4.0], np.float32)


def decode(y):
    """Nearest grid point of a network output."""
    y = np.clip(np.asarray(y, dtype=np.float64), 0.0, 1.0)
    e0 = GRID_EPS[int(np.rint(y[0] * 4))]
    e1 = GRID_EPS[int(np.rint(y[1] * 4))]
    d = GRID_DEPTH[int(np.rint(y[2] * 4))]
    return e0, e1, d


def dataset_matrix(i, count=500, seed=9):
    """Matrix i of the predictor's data set, scaled down from the full-size
    families so an exhaustive sweep fits a few GPU minutes: 7-pt and 27-pt
    stencils (side 12..32), XXZ chains (L = 12..18, even), random geometric
    graphs (3,000..30,000 points, mean degree 20) and random band matrices
    (3,000..30,000 rows, bandwidth 50..500, mean degree ~20)."""
    u = matgen.uniform(3 * count, seed, 0.0, 1.0)
    a, b = u[3 * i], u[3 * i + 1]
    kind = i % 4
    if kind == 0:
        side = 12 + int(a * 21)
        npt = 7 if b < 0.5 else 27
        return f"stencil{npt}_{side}", matgen.stencil3d(side, npt=npt, seed=1000 + i)
    if kind == 1:
        L = 12 + 2 * int(a * 4)
        return f"xxz{L}", matgen.xxz(L)
    if kind == 2:
        n = 3000 + int(a * 27001)
        return f"geometric{n}", matgen.geometric(n, seed=2000 + i)
    n = 3000 + int(a * 27001)
    bw = 50 + int(b * 451)
    return f"banded{n}_{bw}", matgen.banded(n, bw, seed=3000 + i)


def dataset_matrices(count=500, seed=9):
    return [dataset_matrix(i, count, seed) for i in range(count)]


_GPU_LOCK = None


def _init_worker(lock):
    global _GPU_LOCK
    _GPU_LOCK = lock


def _sweep_one(args):
    """Worker: all grid points of matrix i.  Schedules are built on the host
    (in parallel across workers); upload and timing hold the GPU lock, so
    timings never overlap."""
    i, count, reps = args
    import torch
    from . import race_upload
    name, m = dataset_matrix(i, count)
    feats = race_features(m)
    times = np.zeros(len(GRID))
    with _GPU_LOCK:
        xd = torch.rand(m["n"], dtype=torch.float64, device="cuda:0")
        bd = torch.empty_like(xd)
        torch.cuda.synchronize()
    for j, (e0, e1, d) in enumerate(GRID):
        s = race_build(m, SWEEP_WORKERS, eps=(e0, e1, 0.5), max_depth=d, host_only=True, windows=False)
        with _GPU_LOCK:
            race_upload(s)
            symm_spmv_exec(s, RACE_EXEC_LEAF_GROUP, xd, bd)
            e_a = torch.cuda.Event(enable_timing=True)
            e_b = torch.cuda.Event(enable_timing=True)
            e_a.record()
            for _ in range(reps):
                symm_spmv_exec(s, RACE_EXEC_LEAF_GROUP, xd, bd)
            e_b.record()
            torch.cuda.synchronize()
            times[j] = e_a.elapsed_time(e_b) * 1e-3 / reps
            s.free()
    return i, name, feats, times


def sweep(count=500, out_path=None, log=sys.stderr, workers=None, reps=2):
    """Exhaustive grid sweep on the GPU; returns and saves features, times."""
    import multiprocessing as mp
    workers = workers or min(16, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    lock = ctx.Lock()
    feats = np.zeros((count, 16), np.float32)
    times = np.zeros((count, len(GRID)), np.float64)
    names = [""] * count
    t0 = time.time()
    with ctx.Pool(workers, initializer=_init_worker, initargs=(lock,)) as pool:
        for k, (i, name, f, t) in enumerate(pool.imap_unordered(_sweep_one, [(i, count, reps) for i in range(count)])):
            feats[i], times[i], names[i] = f, t, name
            if k % 25 == 0:
                print(f"sweep {k}/{count} {name} best {t.min()*1e6:.1f} us "
                      f"paper {t[point_index(*PAPER_POINT)]*1e6:.1f} us  {time.time()-t0:.0f} s", file=log, flush=True)
    names = np.array(names)
    out_path = out_path or os.path.join(DATA, "predictor_sweep.npz")
    os.makedirs(os.path.dirname(out_path), exist_ok=True)
    np.savez_compressed(out_path, features=feats, times=times, names=names,
                        grid=np.array(GRID, dtype=np.float64), workers=SWEEP_WORKERS)
    return feats, times, names


def split(n, seed=7, n_test=100):
    """400 / 100 train-test split (seed 7)."""
    perm = np.random.default_rng(seed).permutation(n)
    return np.sort(perm[n_test:]), np.sort(perm[:n_test])


class Predictor:
    """The perceptron on the GPU: packed FP32 parameters + Adam state."""

    def __init__(self, seed=0, device="cuda:0"):
        import torch
        self.torch = torch
        self.dev = torch.device(device)
        n = lib().race_mlp_param_count()
        rng = np.random.default_rng(seed)
        p = np.zeros(n, np.float32)
        o = 0
        for fan_in, fan_out in ((16, 64), (64, 64), (64, 3)):
            p[o:o + fan_in * fan_out] = rng.normal(0.0, np.sqrt(2.0 / fan_in), fan_in * fan_out)
            o += fan_in * fan_out + fan_out
        self.params = torch.from_numpy(p).to(self.dev)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.step = 0
        self.mu = np.zeros(16, np.float32)
        self.sd = np.ones(16, np.float32)

    def _norm(self, F):
        return np.ascontiguousarray(((np.asarray(F, np.float32) - self.mu) / self.sd).astype(np.float32))

    def fit(self, F, T, epochs=400, batch=64, lr=2e-3, out_weight=(1.0, 1.0, 1.0), seed=0):
        """Mini-batch Adam on the MSE of the encoded targets; returns the loss history."""
        torch = self.torch
        F = np.asarray(F, np.float32)
        self.mu = F.mean(0)
        self.sd = F.std(0) + 1e-6
        X = torch.from_numpy(self._norm(F)).to(self.dev)
        Y = torch.from_numpy(np.ascontiguousarray(np.asarray(T, np.float32))).to(self.dev)
        w = torch.tensor(out_weight, dtype=torch.float32, device=self.dev)
        n = X.shape[0]
        act = torch.empty(lib().race_mlp_act_size(batch), dtype=torch.float32, device=self.dev)
        work = torch.empty(lib().race_mlp_work_size(batch), dtype=torch.float32, device=self.dev)
        terms = torch.empty(batch * 3, dtype=torch.float32, device=self.dev)
        rng = np.random.default_rng(seed)
        hist = []
        for _ in range(epochs):
            order = rng.permutation(n)
            tot = 0.0
            for s0 in range(0, n - batch + 1, batch):
                idx = torch.from_numpy(order[s0:s0 + batch]).to(self.dev)
                xb = X[idx].contiguous()
                yb = Y[idx].contiguous()
                race_mlp_forward(self.params, batch, xb, act)
                race_mlp_backward(self.params, batch, xb, act, yb, w, self.grad, work, terms)
                self.step += 1
                race_mlp_adam(self.params, self.grad, self.m, self.v, lr, self.step)
                tot += float(terms.sum())
            hist.append(tot / max(1, n // batch))
        return hist

    def predict(self, F):
        torch = self.torch
        X = torch.from_numpy(self._norm(np.atleast_2d(F))).to(self.dev)
        B = X.shape[0]
        act = torch.empty(lib().race_mlp_act_size(B), dtype=torch.float32, device=self.dev)
        y = torch.empty(B * 3, dtype=torch.float32, device=self.dev)
        race_mlp_forward(self.params, B, X, act, y)
        return y.cpu().numpy().reshape(B, 3)

    def choose(self, F):
        """Grid points (eps_0, eps_1, depth) for feature rows F."""
        return [decode(y) for y in self.predict(F)]

    def save(self, path):
        np.concatenate([self.mu, self.sd, self.params.cpu().numpy()]).astype(np.float32).tofile(path)

    def load(self, path):
        a = np.fromfile(path, dtype=np.float32)
        self.mu, self.sd = a[:16].copy(), a[16:32].copy()
        self.params.copy_(self.torch.from_numpy(a[32:].copy()).to(self.dev))
        return self


def regret(times, choice_idx):
    """time at the chosen grid point / best time - 1, per matrix."""
    best = times.min(1)
    return times[np.arange(len(times)), choice_idx] / best - 1.0


def evaluate(pred, feats, times):
    """Mean and median regret of the predictor and of the paper's default point."""
    pts = pred.choose(feats)
    idx = np.array([point_index(*p) for p in pts])
    r_mlp = regret(times, idx)
    r_def = regret(times, np.full(len(times), point_index(*PAPER_POINT)))
    return {"mlp_mean": float(r_mlp.mean()), "mlp_median": float(np.median(r_mlp)),
            "paper_mean": float(r_def.mean()), "paper_median": float(np.median(r_def)),
            "mlp_hits": int(np.sum(r_mlp == 0.0)), "n": int(len(times))}


def labels(times):
    best = times.argmin(1)
    return np.stack([encode(*GRID[j]) for j in best])


def main(argv):
    if argv and argv[0] == "sweep":
        count = int(argv[1]) if len(argv) > 1 else 500
        sweep(count)
    elif argv and argv[0] == "train":
        d = np.load(os.path.join(DATA, "predictor_sweep.npz"))
        feats, times = d["features"], d["times"]
        tr, te = split(len(feats))
        pred = Predictor(seed=0)
        hist = pred.fit(feats[tr], labels(times[tr]))
        pred.save(os.path.join(DATA, "predictor.f32"))
        print({"loss_first": hist[0], "loss_last": hist[-1], **evaluate(pred, feats[te], times[te])})
    else:
        print(__doc__)


if __name__ == "__main__":
    main(sys.argv[1:])
