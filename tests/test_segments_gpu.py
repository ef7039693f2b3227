"""GPU parity of the segmented calls against the CPU oracle (stable per-segment
sort with payload).

Small and mid sizes are compared element by element; the 2^24-segment uneven
batch and the 2^20-segment RSS range run at full size in the bench's launch
configuration and are checked on sampled segments against the oracle plus
sortedness and the Sec. 4.1 permutation product of keys and payload.
"""
import zlib

import numpy as np
import pytest

import oracle
import paper_2002_05599_gb300 as sn
from paper_2002_05599_gb300 import workloads as wl
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

CALLS = {
    ("sn", np.uint32): sn.sn_sort_segments,
    ("sn", np.uint64): sn.sn_sort_segments_u64,
    ("rss", np.uint32): sn.rss_sort_segments,
    ("rss", np.uint64): sn.rss_sort_segments_u64,
}


def run_segments(mode, keys, vals, offsets):
    dtype = keys.dtype.type
    tk, to_ = to_dev(keys), to_dev(offsets)
    tv = to_dev(vals) if vals is not None else None
    sn.check(CALLS[(mode, dtype)](tk, tv, to_))
    sn.check(sn.sn_check())
    return to_host(tk, dtype), (to_host(tv, np.uint32) if tv is not None else None)


def assert_parity(mode, keys, vals, offsets):
    got_k, got_v = run_segments(mode, keys, vals, offsets)
    ref_k, ref_v = oracle.sort_segments(keys, vals, offsets)
    assert np.array_equal(got_k, ref_k)
    if vals is not None:
        assert np.array_equal(got_v, ref_v)


@pytest.mark.parametrize("mode", ["sn", "rss"])
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("with_vals", [True, False])
@pytest.mark.parametrize("lengths,lo,hi", [("uniform", 1, 16), ("geometric", 1, 256), ("uniform", 17, 256)])
def test_segments_parity(mode, dtype, with_vals, lengths, lo, hi):
    for keys in ("uniform", "fewdistinct", "zipf"):
        k, v, off = wl.segment_batch(6000, lengths, keys, dtype, with_vals, seed=zlib.crc32(f"{lengths}{lo}{keys}".encode()) & 0xFFFF,
                                     lo=lo, hi=hi)
        assert_parity(mode, k, v, off)


@pytest.mark.parametrize("mode", ["sn", "rss"])
@pytest.mark.parametrize("lengths,lo,hi", [("uniform", 1, 16), ("geometric", 1, 256), ("uniform", 1, 256)])
def test_segments_many_tiles(mode, lengths, lo, hi):
    # enough segments that every persistent CTA reuses its staging buffers
    # many times (the full-size workloads' steady state), compared in full
    k, v, off = wl.segment_batch(1 << 18, lengths, "uniform", np.uint64, True, seed=21, lo=lo, hi=hi)
    assert_parity(mode, k, v, off)
    k32 = (k >> np.uint64(40)).astype(np.uint32)
    assert_parity(mode, k32, None, off)


@pytest.mark.parametrize("mode", ["sn", "rss"])
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_segments_every_length(mode, dtype):
    # every length 0..256, several of each, shuffled
    rng = np.random.default_rng(3)
    lens = np.repeat(np.arange(0, 257, dtype=np.uint32), 5)
    rng.shuffle(lens)
    off = wl.offsets_from_lengths(lens)
    total = int(off[-1])
    for kind in ("uniform", "fewdistinct"):
        k = wl.uniform_keys(total, dtype, seed=9)
        if kind == "fewdistinct":
            k = k % dtype(3)
        v = np.arange(total, dtype=np.uint32)[::-1].copy()
        assert_parity(mode, k, v, off)
        assert_parity(mode, k, None, off)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("net64", [True, False])
@pytest.mark.parametrize("mode", [0, 1])
def test_segments_33_to_64(dtype, net64, mode):
    # segments of 33..64 items: 64-channel warp network (net_classes bit 4) or
    # Register Sample Sort, after either tile kernel (mode 0 ring, mode 1
    # synchronous); many keys equal to the maximum (the padding value) and
    # many ties; a few short and long segments mixed in
    kb = np.dtype(dtype).itemsize
    rng = np.random.default_rng(21)
    lens = np.concatenate([np.repeat(np.arange(33, 65, dtype=np.uint32), 40),
                           np.array([0, 1, 5, 16, 17, 32, 65, 200, 256] * 5, dtype=np.uint32)])
    rng.shuffle(lens)
    off = wl.offsets_from_lengths(lens)
    total = int(off[-1])
    k = wl.uniform_keys(total, dtype, seed=22)
    k[rng.random(total) < 0.3] = np.iinfo(dtype).max
    k[rng.random(total) < 0.3] = dtype(5)
    v = np.arange(total, dtype=np.uint32)
    try:
        for with_vals in (True, False):
            sn.check(sn.sn_tuning_set(kb, with_vals, net_classes=0x1F if net64 else 0xF, tile_mode=mode), "set")
            assert_parity("sn", k, v if with_vals else None, off)
    finally:
        for with_vals in (True, False):
            sn.check(sn.sn_tuning_set(kb, with_vals), "defaults")


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_segments_edge_cases(dtype):
    top = np.iinfo(dtype).max
    # all-equal, max-key and empty segments, non-zero first offset
    lens = np.array([0, 1, 256, 0, 2, 33, 17, 16, 256, 1, 0], dtype=np.uint32)
    off = wl.offsets_from_lengths(lens) + np.uint32(5)
    total = int(off[-1]) + 3
    k = wl.uniform_keys(total, dtype, seed=4) % dtype(2)
    k[300:560] = top
    v = np.arange(total, dtype=np.uint32)
    for mode in ("sn", "rss"):
        got_k, got_v = run_segments(mode, k, v, off)
        ref_k, ref_v = oracle.sort_segments(k, v, off)
        assert np.array_equal(got_k, ref_k) and np.array_equal(got_v, ref_v)
        assert np.array_equal(got_k[:5], k[:5]) and np.array_equal(got_k[-3:], k[-3:])


def test_segments_all_empty_and_single():
    for lens in (np.zeros(1000, np.uint32), np.ones(5000, np.uint32)):
        off = wl.offsets_from_lengths(lens)
        k = wl.uniform_keys(max(int(off[-1]), 1), np.uint64, seed=2)
        v = np.arange(k.size, dtype=np.uint32)
        assert_parity("sn", k, v, off)


@pytest.mark.parametrize("mode", ["sn", "rss"])
@pytest.mark.parametrize("shift", [1, 2, 3])
def test_segments_misaligned_pointers(mode, shift):
    # keys / vals / offsets `shift` elements past a 16-byte boundary (the plan
    # kernel reads the offsets in aligned 16-byte groups), batches whose last
    # group is cut at every position, and batches of a few segments (only the
    # general path of the plan kernel)
    for nseg in (1, 2, 3, 5, 3000, 3001, 3002, 3003):
        k, v, off = wl.segment_batch(nseg, "geometric", "uniform", np.uint64, True, seed=12 + nseg)
        pad_k = to_dev(np.concatenate([np.zeros(shift, np.uint64), k]))
        pad_v = to_dev(np.concatenate([np.zeros(shift, np.uint32), v]))
        pad_o = to_dev(np.concatenate([np.zeros(shift, np.uint32), off]))
        fn = CALLS[(mode, np.uint64)]
        sn.check(fn(pad_k.data_ptr() + 8 * shift, pad_v.data_ptr() + 4 * shift, pad_o.data_ptr() + 4 * shift,
                    off.size - 1))
        sn.check(sn.sn_check())
        ref_k, ref_v = oracle.sort_segments(k, v, off)
        assert np.array_equal(to_host(pad_k, np.uint64)[shift:], ref_k)
        assert np.array_equal(to_host(pad_v, np.uint32)[shift:], ref_v)


def test_segments_bad_offsets_leave_data_untouched():
    for lens_bad in ("long", "decreasing", "first", "last"):
        k, v, off = wl.segment_batch(2000, "uniform", "uniform", np.uint32, True, seed=8)
        off = off.astype(np.int64)
        if lens_bad == "long":
            off[1000:] += 300  # segment 999 gets 300+ items
        elif lens_bad == "decreasing":
            off[700] = off[699] - 1  # segment 699 gets a negative length
        elif lens_bad == "first":
            off[1:] += 300  # segment 0 (the batch's first offsets group)
        else:
            off[-1] += 300  # the last segment (the batch's last group)
        off = off.astype(np.uint32)
        tk, tv, to_ = to_dev(k), to_dev(v), to_dev(off)
        assert sn.sn_sort_segments(tk, tv, to_) == sn.SN_OK  # detected on the device
        assert sn.sn_check() == sn.SN_ERANGE
        assert np.array_equal(to_host(tk, np.uint32), k)
        assert np.array_equal(to_host(tv, np.uint32), v)
        assert sn.sn_check() == sn.SN_OK  # the status word was cleared


def _sampled_full_check(mode, keys, vals, offsets, nsample=4000):
    tk, tv, to_ = to_dev(keys), to_dev(vals) if vals is not None else None, to_dev(offsets)
    sn.check(CALLS[(mode, keys.dtype.type)](tk, tv, to_))
    sn.check(sn.sn_check())
    got_k = to_host(tk, keys.dtype.type)
    got_v = to_host(tv, np.uint32) if vals is not None else None
    assert oracle.is_sorted_segments(got_k, offsets)
    assert oracle.perm_product(got_k) == oracle.perm_product(keys)
    if vals is not None:
        assert oracle.perm_product(got_v) == oracle.perm_product(vals)
    rng = np.random.default_rng(0)
    nseg = offsets.size - 1
    for s in np.unique(np.concatenate([rng.integers(0, nseg, nsample), [0, nseg - 1]])):
        a, b = int(offsets[s]), int(offsets[s + 1])
        sub_off = np.array([0, b - a], dtype=np.uint32)
        rk, rv = oracle.sort_segments(keys[a:b], None if vals is None else vals[a:b], sub_off)
        assert np.array_equal(got_k[a:b], rk)
        if vals is not None:
            assert np.array_equal(got_v[a:b], rv)


@pytest.mark.parametrize("lengths", ["uniform", "geometric"])
def test_uneven_batch_full_size(lengths):
    # 2^24 segments, u64 keys uniform, u32 payload = original index
    k, v, off = wl.segment_batch(1 << 24, lengths, "uniform", np.uint64, True, seed=1, lo=1, hi=16)
    _sampled_full_check("sn", k, v, off)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("keys", ["uniform", "zipf"])
def test_rss_range_full_size(dtype, keys):
    # 2^20 segments of 17..256 items, keys only
    k, _, off = wl.segment_batch(1 << 20, "uniform", keys, dtype, False, seed=1, lo=17, hi=256)
    _sampled_full_check("rss", k, None, off)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_segments_window_ties_take_the_exact_path(dtype):
    # Payload sorts run their networks on composites of a key window and the
    # item's slot.  Keys built to differ in their top bit and in their lowest
    # bits only make two different keys share a window, so the networks' tie
    # check must send those segments through the exact fallback; keys equal
    # in all bits must still keep their input order.
    rng = np.random.default_rng(51)
    bits = 8 * np.dtype(dtype).itemsize
    for lo, hi in ((2, 16), (17, 32), (33, 64), (2, 256)):
        k, v, off = wl.segment_batch(20000, "uniform", "uniform", dtype, True, seed=52 + lo, lo=lo, hi=hi)
        top = (rng.integers(0, 2, k.size).astype(np.uint64) << np.uint64(bits - 1))
        low = rng.integers(0, 4, k.size).astype(np.uint64)
        k = (top | low).astype(dtype)
        for mode in ("sn", "rss"):
            assert_parity(mode, k, v, off)
            assert_parity(mode, k, None, off)
