"""GPU parity of the Bose-Nelson network family and of the paper's 16-byte
items (u64 key + u64 reference, Sec. 4.1) against the CPU oracle.

Bit-exact for every n = 2..16 at sizes spanning several tiles plus a ragged
tail, for both network families, with many equal keys (items must keep their
order among equal keys), on 16-byte-aligned (bulk-copy) and 8-byte-aligned
(direct) buffers.
"""
import numpy as np
import pytest

import oracle
import paper_2002_05599_gb300 as sn
from paper_2002_05599_gb300 import workloads as wl
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu
FAMILIES = [sn.SN_NETWORK_BEST, sn.SN_NETWORK_BOSE_NELSON]


@pytest.mark.parametrize("dist", ["uniform", "fewdistinct", "reverse"])
def test_bose_nelson_family_u32_all_n(dist):
    for n in range(2, 17):
        keys = wl.fixed_arrays(n, 5 * 2048 + 19, dist, np.uint32, seed=300 + n)
        t = to_dev(keys)
        sn.check(sn.sn_sort_fixed_family(t, n, sn.SN_NETWORK_BOSE_NELSON), f"n={n}")
        sn.check(sn.sn_check())
        assert np.array_equal(to_host(t, np.uint32), oracle.sort_fixed(keys, n)), f"n={n}"


def _items(count, n, seed, distinct=8):
    rng = np.random.default_rng(seed)
    items = np.empty(2 * count * n, np.uint64)
    items[0::2] = rng.integers(0, distinct, count * n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    items[1::2] = rng.integers(0, 2**63, count * n, dtype=np.uint64)
    return items


@pytest.mark.parametrize("family", FAMILIES)
def test_items_all_n(family):
    for n in range(2, 17):
        count = 3 * 512 + 11  # several tiles (256 or 512 arrays each) and a ragged tail
        items = _items(count, n, seed=400 + n)
        t = to_dev(items)
        sn.check(sn.sn_sort_fixed_items(t, n, family), f"n={n}")
        sn.check(sn.sn_check())
        assert np.array_equal(to_host(t, np.uint64), oracle.sort_fixed_items(items, n)), f"n={n}"


@pytest.mark.parametrize("family", FAMILIES)
def test_items_unaligned_and_small(family):
    import torch
    for n in (3, 8, 16):
        for count in (1, 7, 300):
            items = _items(count, n, seed=n * count)
            buf = torch.zeros(items.size + 1, dtype=torch.int64, device="cuda")
            view = buf[1:]  # 8-byte aligned, not 16: the direct path
            view.copy_(to_dev(items))
            sn.check(sn.sn_sort_fixed_items(view, n, family, count=count))
            sn.check(sn.sn_check())
            assert np.array_equal(to_host(view.contiguous(), np.uint64), oracle.sort_fixed_items(items, n))


def test_family_and_item_argument_errors():
    import torch
    t = torch.zeros(64, dtype=torch.int32, device="cuda")
    assert sn.sn_sort_fixed_family(t, 8, 2) == sn.SN_EINVAL
    assert sn.sn_sort_fixed_family(t, 17, sn.SN_NETWORK_BEST) == sn.SN_EINVAL
    it = torch.zeros(64, dtype=torch.int64, device="cuda")
    assert sn.sn_sort_fixed_items(it, 8, 5) == sn.SN_EINVAL
    assert sn.sn_sort_fixed_items(it, 1, sn.SN_NETWORK_BEST) == sn.SN_EINVAL
