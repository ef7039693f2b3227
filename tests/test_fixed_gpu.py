"""GPU parity of sn_sort_fixed / sn_sort_fixed_u64 against the CPU oracle.

Bit-exact on the seeded inputs of every distribution for n = 2..16, at sizes
that span several tiles plus a ragged tail; edge cases (count 0/1, one partial
tile, misaligned keys, maximum key values); the 2^20-array n = 8 workload in
full; and the 2^24-array sweep workload in the bench's launch configuration,
checked on sampled arrays against the oracle plus sortedness and the
Sec. 4.1 permutation product on every array.
"""
import numpy as np
import pytest

import oracle
import paper_2002_05599_gb300 as sn
from paper_2002_05599_gb300 import workloads as wl
from gpu_util import row_products, rows_sorted, to_dev, to_host

pytestmark = pytest.mark.gpu

FN = {np.uint32: sn.sn_sort_fixed, np.uint64: sn.sn_sort_fixed_u64}


def run_fixed(keys, n, dtype):
    t = to_dev(keys)
    sn.check(FN[dtype](t, n))
    sn.check(sn.sn_check())
    return to_host(t, dtype)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("dist", ["uniform", "fewdistinct", "presorted", "reverse"])
def test_fixed_parity_all_n(dtype, dist):
    for n in range(2, 17):
        count = 9 * 2048 + 37  # several tiles for every n, plus a ragged tail
        keys = wl.fixed_arrays(n, count, dist, dtype, seed=100 + n)
        got = run_fixed(keys, n, dtype)
        assert np.array_equal(got, oracle.sort_fixed(keys, n)), f"n={n}"


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("count", [1, 2, 31, 255, 256, 257, 4095])
def test_fixed_small_counts(dtype, count):
    for n in (2, 3, 8, 13, 16):
        keys = wl.fixed_arrays(n, count, "uniform", dtype, seed=count + n)
        assert np.array_equal(run_fixed(keys, n, dtype), oracle.sort_fixed(keys, n))


def test_fixed_count_zero_is_noop():
    import torch
    t = torch.arange(16, dtype=torch.int32, device="cuda")
    assert sn.sn_sort_fixed(t, 8, 0) == sn.SN_OK
    assert torch.equal(t.cpu(), torch.arange(16, dtype=torch.int32))


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_fixed_max_keys(dtype):
    top = np.iinfo(dtype).max
    for n in (4, 9, 16):
        keys = wl.fixed_arrays(n, 3000, "fewdistinct", dtype, seed=n)
        keys = np.where(keys == 0, dtype(top), keys).astype(dtype)
        assert np.array_equal(run_fixed(keys, n, dtype), oracle.sort_fixed(keys, n))


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_fixed_misaligned_keys(dtype):
    for n in (3, 8, 16):
        count = 5000
        keys = wl.fixed_arrays(n, count, "uniform", dtype, seed=7 * n)
        buf = to_dev(np.concatenate([np.zeros(1, dtype), keys, np.zeros(1, dtype)]))
        base = buf.data_ptr() + buf.element_size()  # one element past a 16-byte boundary
        sn.check(FN[dtype](base, n, count))
        sn.check(sn.sn_check())
        out = to_host(buf, dtype)
        assert out[0] == 0 and out[-1] == 0
        assert np.array_equal(out[1:-1], oracle.sort_fixed(keys, n))


def test_fixed_config_n8_full():
    # 2^20 arrays of 8 uniform u32 keys from seed 1, compared in full
    n, count = 8, 1 << 20
    keys = wl.fixed_arrays(n, count, "uniform", np.uint32, seed=1)
    assert np.array_equal(run_fixed(keys, n, np.uint32), oracle.sort_fixed(keys, n))


@pytest.mark.parametrize("n", [2, 5, 8, 12, 16])
def test_fixed_sweep_full_size_sampled(n):
    # 2^24 arrays (the sweep workload), as the benchmark launches it
    import torch
    count = 1 << 24
    keys = wl.fixed_arrays(n, count, "uniform", np.uint32, seed=1)
    t = to_dev(keys)
    before = row_products(t, n)
    sn.check(sn.sn_sort_fixed(t, n))
    sn.check(sn.sn_check())
    assert rows_sorted(t, n)
    assert torch.equal(row_products(t, n), before)
    rng = np.random.default_rng(n)
    idx = np.unique(np.concatenate([rng.integers(0, count, 65536), [0, count - 1]]))
    got = t.view(-1, n)[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint32)
    want = oracle.sort_fixed(keys.reshape(-1, n)[idx].reshape(-1), n).reshape(-1, n)
    assert np.array_equal(got, want)
