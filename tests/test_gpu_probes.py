"""The diagnostic ceilings of the roofline (race_probe_peaks): the load-only
stream reads every word once (its XOR fold matches the host's), the FP64
fused multiply-add chains run, and malformed requests are refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1907_06487_gb300 as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06487_gb300 import build
    build.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("n", [1, 2, 7, 1000, 1 << 20, (1 << 20) + 3])
def test_load_stream_reads_every_word(dev, n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n)
    inp = torch.from_numpy(a).to(dev)
    out = torch.zeros(4096, dtype=torch.float64, device=dev)
    R.race_probe_peaks(0, inp, n, out)
    torch.cuda.synchronize()
    blocks = torch.cuda.get_device_properties(dev).multi_processor_count * 4
    got = np.bitwise_xor.reduce(out.cpu().numpy()[:blocks].view(np.uint64))
    want = np.bitwise_xor.reduce(a.view(np.uint64))
    assert got == want


def test_fma_chains_and_refusals(dev):
    out = torch.zeros(4096, dtype=torch.float64, device=dev)
    R.race_probe_peaks(1, None, 0, out, 64)
    torch.cuda.synchronize()
    blocks = torch.cuda.get_device_properties(dev).multi_processor_count * 4
    assert np.all(np.isfinite(out.cpu().numpy()[:blocks])) and float(out[0]) > 0
    inp = torch.zeros(9, dtype=torch.float64, device=dev)
    for args in ((0, inp[1:], 8, out, 1), (1, None, 0, out, 0), (2, inp, 8, out, 1), (0, inp, -1, out, 1)):
        with pytest.raises(R.RaceError) as e:
            R.race_probe_peaks(*args)
        assert e.value.code == R.RACE_ERR_INVALID


def test_reduction_paths_count_every_contribution(dev):
    """race_probe_reductions: reductions at L2 and bulk row reductions count
    every index exactly; a plain read-modify-write does too when no index
    repeats; the shared and cluster-shared atomics lose none (all indices on
    slot 0: the blocks' slot-0 totals sum to m)."""
    rng = np.random.default_rng(3)
    n, m = 5000, 200000
    idx = rng.integers(0, n, m).astype(np.int32)
    idx_d = torch.from_numpy(idx).to(dev)
    want = np.bincount(idx, minlength=n).astype(np.float64)
    t = torch.zeros(16 * n, dtype=torch.float64, device=dev)
    R.race_probe_reductions(0, idx_d, m, n - 1, t, n)
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy()[:n], want)
    t.zero_()
    R.race_probe_reductions(4, idx_d, m, n - 1, t, 16 * n)
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy().reshape(n, 16), np.repeat(want[:, None], 16, 1))
    perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).to(dev)
    t.zero_()
    R.race_probe_reductions(1, perm, n, n - 1, t, n)
    torch.cuda.synchronize()
    assert np.all(t.cpu().numpy()[:n] == 1.0)
    zeros = torch.zeros(m, dtype=torch.int32, device=dev)
    blocks = torch.cuda.get_device_properties(dev).multi_processor_count * 8
    for mode in (2, 3):
        t.zero_()
        R.race_probe_reductions(mode, zeros, m, n - 1, t, max(n, blocks))
        torch.cuda.synchronize()
        assert float(t[:blocks].sum()) == float(m), mode
    with pytest.raises(R.RaceError):
        R.race_probe_reductions(4, idx_d, m, n - 1, t, n)  # target too small for rows of 16
    with pytest.raises(R.RaceError):
        R.race_probe_reductions(5, idx_d, m, n - 1, t, n)
