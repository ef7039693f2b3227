"""GPU parity of the float32 / float64 calls against the CPU oracle (IEEE 754
totalOrder), bit for bit: random bit patterns (so NaNs of both signs with
many payloads, infinities, signed zeros and subnormals all occur), plus a
dense mix of the special values, for fixed n = 2..16 and for CSR segments of
0..256 keys with and without payload."""
import numpy as np
import pytest

import oracle
import paper_2002_05599_gb300 as sn
from paper_2002_05599_gb300 import workloads as wl
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

SPECIAL32 = [0x7FC00000, 0xFFC00000, 0x7F800001, 0xFFBFFFFF, 0x80000000, 0, 0x7F800000, 0xFF800000, 1, 0x80000001]
SPECIAL64 = [0x7FF8000000000000, 0xFFF8000000000000, 0x8000000000000000, 0, 0x7FF0000000000000,
             0xFFF0000000000000, 1, 0x8000000000000001, 0x7FF0000000000001]


def _float_keys(count, dtype, seed):
    u = np.uint32 if dtype == np.float32 else np.uint64
    bits = wl.uniform_keys(count, u, seed)
    rng = np.random.default_rng(seed)
    special = SPECIAL32 if dtype == np.float32 else SPECIAL64
    pick = rng.random(count) < 0.25
    bits[pick] = np.array(special, dtype=u)[rng.integers(0, len(special), int(pick.sum()))]
    # a quarter ordinary small numbers with repeats
    ordinary = rng.random(count) < 0.25
    bits[ordinary] = (rng.integers(-4, 4, int(ordinary.sum())).astype(dtype) * dtype(0.5)).view(u)
    return bits.view(dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_fixed_float_all_n(dtype):
    fn = sn.sn_sort_fixed_f32 if dtype == np.float32 else sn.sn_sort_fixed_f64
    u = np.uint32 if dtype == np.float32 else np.uint64
    for n in range(2, 17):
        keys = _float_keys(n * (4 * 2048 + 13), dtype, seed=600 + n)
        t = to_dev(keys.view(u))
        sn.check(fn(t, n), f"n={n}")
        sn.check(sn.sn_check())
        assert np.array_equal(to_host(t, u), oracle.sort_fixed(keys, n).view(u)), f"n={n}"


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("with_vals", [False, True])
@pytest.mark.parametrize("lengths", ["uniform", "geometric"])
def test_segments_float(dtype, with_vals, lengths):
    fn = sn.sn_sort_segments_f32 if dtype == np.float32 else sn.sn_sort_segments_f64
    u = np.uint32 if dtype == np.float32 else np.uint64
    _, v, off = wl.segment_batch(40_000, lengths, "uniform", u, with_vals, seed=61, lo=0, hi=256)
    keys = _float_keys(int(off[-1]), dtype, seed=62)
    ek, ev = oracle.sort_segments(keys, v, off)
    dk = to_dev(keys.view(u))
    dv = to_dev(v) if with_vals else None
    sn.check(fn(dk, dv, to_dev(off)))
    sn.check(sn.sn_check())
    assert np.array_equal(to_host(dk, u), ek.view(u))
    if with_vals:
        assert np.array_equal(to_host(dv, np.uint32), ev)
