"""GPU parity of sn_sort_segments_large(_u64) (segments of up to 4096 items)
against the CPU oracle, and its device-side validation."""
import numpy as np
import pytest

import oracle
import paper_2002_05599_gb300 as sn
from paper_2002_05599_gb300 import workloads as wl
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


def _batch(nseg, dtype, with_vals, seed, keys="uniform"):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, 4097, nseg).astype(np.uint32)
    lens[::5] = rng.integers(0, 40, lens[::5].size)      # short segments mixed in
    lens[3::11] = 4096                                    # the maximum
    off = wl.offsets_from_lengths(lens)
    total = int(off[-1])
    k = wl.uniform_keys(total, dtype, seed)
    if keys == "fewdistinct":
        k = k % dtype(3)
    v = np.arange(total, dtype=np.uint32) if with_vals else None
    return k, v, off


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("with_vals", [False, True])
@pytest.mark.parametrize("keys", ["uniform", "fewdistinct"])
def test_large_segments_match_oracle(dtype, with_vals, keys):
    fn = sn.sn_sort_segments_large if dtype == np.uint32 else sn.sn_sort_segments_large_u64
    k, v, off = _batch(120, dtype, with_vals, seed=71 + int(with_vals), keys=keys)
    ek, ev = oracle.sort_segments(k, v, off)
    dk = to_dev(k)
    dv = to_dev(v) if with_vals else None
    sn.check(fn(dk, dv, to_dev(off)))
    assert sn.sn_check() == sn.SN_OK
    assert np.array_equal(to_host(dk, dtype), ek)
    if with_vals:
        assert np.array_equal(to_host(dv, np.uint32), ev)


def test_large_rejects_long_or_decreasing_offsets():
    for off in (np.array([0, 10, 4107, 4110], np.uint32), np.array([0, 10, 5, 20], np.uint32)):
        k = wl.uniform_keys(int(off.max()), np.uint32, 3)
        dk = to_dev(k)
        sn.check(sn.sn_sort_segments_large(dk, None, to_dev(off)))
        assert sn.sn_check() == sn.SN_ERANGE
        assert np.array_equal(to_host(dk, np.uint32), k)  # untouched
