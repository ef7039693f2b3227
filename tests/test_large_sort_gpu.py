"""GPU parity of sn_sort_large (one large u32 array: sample-sort partition
with the segmented sort as base case) against the oracle's merge sort, over
sizes that take the single-segment path, one partition level, and a
recursively sorted sample, and over distributions with heavy duplicates."""
import numpy as np
import pytest

import oracle
import paper_2002_05599_gb300 as sn
from paper_2002_05599_gb300 import workloads as wl
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


def _keys(n, dist, seed):
    k = wl.uniform_keys(n, np.uint32, seed)
    if dist == "fewdistinct":
        return k % np.uint32(4)
    if dist == "equal":
        return np.full(n, 7, np.uint32)
    if dist == "sorted":
        return np.sort(k)
    if dist == "reverse":
        return np.sort(k)[::-1].copy()
    if dist == "zipf":
        return wl.zipf_keys(n, dtype=np.uint32, seed=seed)
    return k


@pytest.mark.parametrize("n", [0, 1, 2, 100, 4096, 4097, 65_537, 1_000_003, (1 << 24) + 5])
def test_large_sort_sizes(n):
    k = _keys(n, "uniform", n)
    t = to_dev(k)
    sn.check(sn.sn_sort_large(t))
    assert sn.sn_check() == sn.SN_OK
    assert np.array_equal(to_host(t, np.uint32), oracle.sort_array(k))


@pytest.mark.parametrize("dist", ["fewdistinct", "equal", "sorted", "reverse", "zipf"])
def test_large_sort_distributions(dist):
    n = 3_000_017
    k = _keys(n, dist, 5)
    t = to_dev(k)
    sn.check(sn.sn_sort_large(t))
    assert sn.sn_check() == sn.SN_OK
    assert np.array_equal(to_host(t, np.uint32), oracle.sort_array(k))
