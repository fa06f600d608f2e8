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
The exhaustive sweep stays both the fallback and the measure of the
predictor's regret.

A second data set (dataset_matrix_v2, full sizes: stencils of side 16..128,
XXZ L = 16..24, geometric and band matrices of 10^4..10^6 rows) is swept over
GRID_V2 with the executors that run all rows at once (the library's default)
and one leaf per block, N_t = 152; a network is trained per executor.  Every
evaluation reports the paper's default point and the best single fixed grid
point chosen on the training matrices beside the network.

Usage (GPU):  python -m paper_1907_06487_gb300.predictor sweep        (data/predictor_sweep.npz)
              python -m paper_1907_06487_gb300.predictor train        (data/predictor.f32)
              python -m paper_1907_06487_gb300.predictor sweep_full   (data/predictor_sweep_full.npz)
              python -m paper_1907_06487_gb300.predictor sweep_full_phased (adds the phase-by-phase labels)
              python -m paper_1907_06487_gb300.predictor train_full   (data/predictor_full_*.f32)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

from . import RACE_EXEC_LEAF_GROUP, lib, matgen, race_build, race_features, symm_spmv_exec
from . import race_mlp_adam, race_mlp_backward, race_mlp_forward

class Grid:
    """A grid of schedule parameters (eps_0, eps_1, depth), eps_s = 0.5 for
    s > 1; depth -1 = as deep as the epsilon rule goes (the paper)."""

    def __init__(self, eps, depth):
        self.eps, self.depth = tuple(eps), tuple(depth)
        self.points = [(e0, e1, d) for e0 in self.eps for e1 in self.eps for d in self.depth]

    def __len__(self):
        return len(self.points)

    def index(self, e0, e1, d):
        return self.points.index((e0, e1, d))

    def encode(self, e0, e1, d):
        """Target in [0,1]^3 for a grid point."""
        ne, nd = len(self.eps) - 1, len(self.depth) - 1
        return np.array([self.eps.index(e0) / ne, self.eps.index(e1) / ne, self.depth.index(d) / nd], np.float32)

    def decode(self, y):
        """Nearest grid point of a network output."""
        y = np.clip(np.asarray(y, dtype=np.float64), 0.0, 1.0)
        ne, nd = len(self.eps) - 1, len(self.depth) - 1
        return (self.eps[int(np.rint(y[0] * ne))], self.eps[int(np.rint(y[1] * ne))],
                self.depth[int(np.rint(y[2] * nd))])


# the scaled-down data set, labelled with the schedule-bound executor
GRID_V1 = Grid((0.5, 0.6, 0.7, 0.8, 0.9), (1, 2, 3, 4, -1))
GRID_EPS, GRID_DEPTH, GRID = GRID_V1.eps, GRID_V1.depth, GRID_V1.points
PAPER_POINT = (0.8, 0.8, -1)
SWEEP_WORKERS = 128
HERE = os.path.dirname(os.path.abspath(__file__))
DATA = os.path.join(HERE, "data")


def point_index(e0, e1, d):
    return GRID_V1.index(e0, e1, d)


def encode(e0, e1, d):
    return GRID_V1.encode(e0, e1, d)


def decode(y):
    return GRID_V1.decode(y)


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


# the data set at the sizes of the paper-shaped families, labelled with the
# executors that run all rows at once (the library's default) and one leaf per
# block (the conflict-free one), N_t = 152 as in the benchmark's schedules
GRID_V2 = Grid((0.5, 0.65, 0.8, 0.9), (1, 2, 3, -1))
SWEEP_WORKERS_V2 = 152
V2_LAUNCH = {"default": dict(executor=8, group_lanes=1, rows_per_group=1, blocks_per_sm=0, regs_per_row=4,
                             fp64_quarters=2),
             "leafcta": dict(executor=1, group_lanes=1, rows_per_group=1, blocks_per_sm=0, regs_per_row=8)}
# a third label set, added to the same data set later: the default arithmetic
# run phase by phase (RACE_EXEC_PHASE_DF64), where the number of phases counts
V2_LAUNCH_PHASED = {"phased": dict(executor=13, group_lanes=1, rows_per_group=1, blocks_per_sm=0, regs_per_row=4,
                                   fp64_quarters=2)}


def dataset_matrix_v2(i, count=500, seed=10):
    """Matrix i of the full-size data set: 7-pt and 27-pt stencils of side
    16..128, XXZ chains L = 16..24 (even), random geometric graphs and random
    band matrices (bandwidth 50..500) of 10^4..10^6 rows, mean degree 20;
    sizes log-uniform."""
    u = matgen.uniform(3 * count, seed, 0.0, 1.0)
    a, b = u[3 * i], u[3 * i + 1]
    kind = i % 4
    if kind == 0:
        side = int(round(16 * 8.0 ** a))
        npt = 7 if b < 0.5 else 27
        return f"stencil{npt}_{side}", matgen.stencil3d(side, npt=npt, seed=1000 + i)
    if kind == 1:
        L = 16 + 2 * min(4, int(a * 5))
        return f"xxz{L}", matgen.xxz(L)
    n = int(10.0 ** (4.0 + 2.0 * a))
    if kind == 2:
        return f"geometric{n}", matgen.geometric(n, seed=2000 + i)
    bw = 50 + int(b * 451)
    return f"banded{n}_{bw}", matgen.banded(n, bw, seed=3000 + i)


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


def _sweep_one_v2(args):
    """Worker: every point of GRID_V2 for matrix i, timed with each of the
    given launches (depth-1 points share one schedule across eps_1, which
    stage 0 ignores)."""
    i, count, reps, launches = args
    import torch
    from . import race_set_launch, race_upload, symm_spmv
    name, m = dataset_matrix_v2(i, count)
    feats = race_features(m)
    out = {k: np.zeros(len(GRID_V2)) for k in launches}
    with _GPU_LOCK:
        xd = torch.rand(m["n"], dtype=torch.float64, device="cuda:0")
        bd = torch.empty_like(xd)
        torch.cuda.synchronize()
    done = {}
    for j, (e0, e1, d) in enumerate(GRID_V2.points):
        key = (e0, e1 if d != 1 else None, d)
        if key in done:
            for k in launches:
                out[k][j] = out[k][done[key]]
            continue
        done[key] = j
        s = race_build(m, SWEEP_WORKERS_V2, eps=(e0, e1, 0.5), max_depth=d, host_only=True, windows=False)
        with _GPU_LOCK:
            race_upload(s)
            for k, launch in launches.items():
                race_set_launch(s, 0, **launch)
                # one timed call sizes the repetitions: about 1 ms of work per point,
                # at least `reps` calls, so that short kernels are not launch noise
                e_a = torch.cuda.Event(enable_timing=True)
                e_b = torch.cuda.Event(enable_timing=True)
                symm_spmv(s, xd, bd)
                e_a.record()
                symm_spmv(s, xd, bd)
                e_b.record()
                torch.cuda.synchronize()
                one = max(1e-6, e_a.elapsed_time(e_b) * 1e-3)
                r = int(min(400, max(reps, 1e-3 / one)))
                e_a = torch.cuda.Event(enable_timing=True)
                e_b = torch.cuda.Event(enable_timing=True)
                e_a.record()
                for _ in range(r):
                    symm_spmv(s, xd, bd)
                e_b.record()
                torch.cuda.synchronize()
                out[k][j] = e_a.elapsed_time(e_b) * 1e-3 / r
            s.free()
    return i, name, feats, out


def sweep_v2(count=500, out_path=None, log=sys.stderr, workers=None, reps=6, launches=None, add=False):
    """Full-size sweep over GRID_V2, each point timed with every launch of
    `launches` (default: V2_LAUNCH); saves features and times_<label> arrays.
    add=True keeps the arrays already in the file (same matrices and grid)
    and adds the new labels to it."""
    import multiprocessing as mp
    launches = launches or V2_LAUNCH
    workers = workers or min(16, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    lock = ctx.Lock()
    feats = np.zeros((count, 16), np.float32)
    times = {k: np.zeros((count, len(GRID_V2)), np.float64) for k in launches}
    names = [""] * count
    t0 = time.time()
    with ctx.Pool(workers, initializer=_init_worker, initargs=(lock,)) as pool:
        jobs = [(i, count, reps, launches) for i in range(count)]
        for c, (i, name, f, t) in enumerate(pool.imap_unordered(_sweep_one_v2, jobs)):
            feats[i], names[i] = f, name
            for k in launches:
                times[k][i] = t[k]
            if c % 25 == 0:
                best = "  ".join(f"{k} best {t[k].min()*1e6:.1f} us" for k in launches)
                print(f"sweep_v2 {c}/{count} {name} {best}  {time.time()-t0:.0f} s", file=log, flush=True)
    out_path = out_path or os.path.join(DATA, "predictor_sweep_full.npz")
    os.makedirs(os.path.dirname(out_path), exist_ok=True)
    arrays = {}
    if add and os.path.exists(out_path):
        old = np.load(out_path)
        arrays = {k: old[k] for k in old.files}
        if not (np.array_equal(arrays["names"], np.array(names)) and
                np.array_equal(arrays["grid"], np.array(GRID_V2.points, dtype=np.float64))):
            raise ValueError("sweep_v2(add=True): the file holds another data set or grid")
    arrays.update(features=feats, names=np.array(names), grid=np.array(GRID_V2.points, dtype=np.float64),
                  workers=SWEEP_WORKERS_V2, **{"times_" + k: v for k, v in times.items()})
    np.savez_compressed(out_path, **arrays)
    return feats, times, names


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

    def __init__(self, seed=0, device="cuda:0", grid=None):
        import torch
        self.torch = torch
        self.grid = grid or GRID_V1
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
        return [self.grid.decode(y) for y in self.predict(F)]

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


def best_fixed_point(times, grid=None):
    """The single grid point with the least mean regret over the given
    (training) matrices: the baseline a learned choice has to beat."""
    r = times / times.min(1, keepdims=True) - 1.0
    return (grid or GRID_V1).points[int(np.argmin(r.mean(0)))]


def evaluate(pred, feats, times, fixed=None):
    """Mean and median regret of the predictor, of the paper's default point
    and (if given) of a fixed grid point chosen on the training matrices."""
    g = pred.grid
    pts = pred.choose(feats)
    idx = np.array([g.index(*p) for p in pts])
    r_mlp = regret(times, idx)
    r_def = regret(times, np.full(len(times), g.index(*PAPER_POINT)))
    out = {"mlp_mean": float(r_mlp.mean()), "mlp_median": float(np.median(r_mlp)),
           "paper_mean": float(r_def.mean()), "paper_median": float(np.median(r_def)),
           "mlp_hits": int(np.sum(r_mlp == 0.0)), "n": int(len(times))}
    if fixed is not None:
        r_fix = regret(times, np.full(len(times), g.index(*fixed)))
        out.update({"fixed_point": list(fixed), "fixed_mean": float(r_fix.mean()),
                    "fixed_median": float(np.median(r_fix))})
    return out


def labels(times, grid=None):
    g = grid or GRID_V1
    best = times.argmin(1)
    return np.stack([g.encode(*g.points[j]) for j in best])


def train_and_evaluate(feats, times, grid, seed=0, epochs=400):
    """Train on the 400-matrix split, evaluate on the 100 held out (split
    seed 7): the network, the paper's default and the best fixed point."""
    tr, te = split(len(feats))
    pred = Predictor(seed=seed, grid=grid)
    hist = pred.fit(feats[tr], labels(times[tr], grid), epochs=epochs)
    res = evaluate(pred, feats[te], times[te], best_fixed_point(times[tr], grid))
    return pred, {"loss_first": hist[0], "loss_last": hist[-1], **res}


def main(argv):
    if argv and argv[0] == "sweep":
        count = int(argv[1]) if len(argv) > 1 else 500
        sweep(count)
    elif argv and argv[0] == "sweep_full":
        count = int(argv[1]) if len(argv) > 1 else 500
        sweep_v2(count)
    elif argv and argv[0] == "sweep_full_phased":
        count = int(argv[1]) if len(argv) > 1 else 500
        sweep_v2(count, launches=V2_LAUNCH_PHASED, add=True)
    elif argv and argv[0] == "train":
        d = np.load(os.path.join(DATA, "predictor_sweep.npz"))
        pred, res = train_and_evaluate(d["features"], d["times"], GRID_V1)
        pred.save(os.path.join(DATA, "predictor.f32"))
        print(res)
    elif argv and argv[0] == "train_full":
        d = np.load(os.path.join(DATA, "predictor_sweep_full.npz"))
        for target in [k[len("times_"):] for k in d.files if k.startswith("times_")]:
            pred, res = train_and_evaluate(d["features"], d["times_" + target], GRID_V2)
            pred.save(os.path.join(DATA, f"predictor_full_{target}.f32"))
            print(target, res)
    else:
        print(__doc__)


if __name__ == "__main__":
    main(sys.argv[1:])
