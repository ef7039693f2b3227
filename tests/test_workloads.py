"""The seeded input generators: the torch versions (used to build full-size
bench inputs on the device) produce exactly the numpy versions' values."""
import numpy as np

from paper_2002_05599_gb300 import workloads as wl


def test_uniform_keys_torch_matches_numpy():
    for dt in (np.uint32, np.uint64):
        a = wl.uniform_keys(50_000, dt, seed=3, start=17)
        b = wl.uniform_keys_torch(50_000, dt, seed=3, start=17, device="cpu").numpy()
        assert np.array_equal(a, b.view(dt))


def test_zipf_keys_torch_matches_numpy():
    for dt in (np.uint32, np.uint64):
        a = wl.zipf_keys(80_000, dtype=dt, seed=4)
        b = wl.zipf_keys_torch(80_000, dtype=dt, seed=4, device="cpu").numpy()
        assert np.array_equal(a, b.view(dt))


def test_zipf_keys_are_heavy_tailed_over_2_20_values():
    k = wl.zipf_keys(200_000, seed=5)
    assert k.max() < (1 << 20)
    counts = np.bincount(k, minlength=16)
    # rank r has probability r^-1.1 / H, H = sum over r <= 2^20 of r^-1.1 (about 8.08)
    h = float(np.sum(np.arange(1, (1 << 20) + 1, dtype=np.float64) ** -1.1))
    for r in (1, 2, 4, 8):
        expect = r ** -1.1 / h
        assert abs(counts[r - 1] / k.size - expect) < 4 * np.sqrt(expect / k.size)
