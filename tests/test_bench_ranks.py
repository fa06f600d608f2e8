"""The host logic of bench.py on CPU: two gloo ranks (the N > 1
path runs independent replicas, so its only exchange is the max over ranks
of the timings), the whole-job throughput, and the reference arm's rule that
ranks other than 0 exit without work; and the reference arm's JSON line."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = [0.5 + rank, 2.0 - rank, 3.0 * (rank + 1)]
    got = bench.max_over_ranks(mine, world, "cpu")
    rate = bench.whole_job_rate(world, 1e9, 10, got[0])
    q.put((rank, got, rate))
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in res:
        assert got == [1.5, 2.0, 6.0]              # element-wise max over the ranks
        assert rate == pytest.approx(2 * 1e9 * 10 / 1.5)  # both replicas' work over the slowest time


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([1.0, 2.0], 1, "cpu") == [1.0, 2.0]
    assert bench.whole_job_rate(1, 5.0, 4, 2.0) == 10.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.build_parser().parse_args(["--impl", "reference", "--gpus", "2"])
    assert bench.run_reference(args) == 0


def test_reference_arm_line(tmp_path):
    """bench.py --impl reference on one process: one JSON line with the
    contract's keys, the oracle timed on the host cores under our arm's metric
    name, no host-device bytes (CPU only)."""
    import json
    import subprocess
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "anderson32", "--steps", "3", "--warmup", "3", "--ref-seconds", "1"],
                         capture_output=True, text=True, env=env, cwd=str(tmp_path), timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC_SYMM
    for key in ("value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "GFLOP/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == "anderson32"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
