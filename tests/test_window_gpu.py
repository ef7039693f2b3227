"""GPU parity of the one-launch window path of the segmented calls (launch
parameter tile_mode 2) against the CPU oracle, under several window
capacities and staging depths: every length 0..256, payload or not, u32 / u64
/ float keys, RSS-only mode, the 64-item network on and off, misaligned
pointers, a batch big enough that every warp cycles through its buffers many
times, and bad offsets (the batch stays untouched)."""
import numpy as np
import pytest

import oracle
import paper_2002_05599_gb300 as sn
from paper_2002_05599_gb300 import workloads as wl
from gpu_util import to_dev, to_host
from test_segments_gpu import assert_parity, run_segments

pytestmark = pytest.mark.gpu

# (window capacity in items, windows in flight per warp)
WINDOWS = [(512, 2), (1024, 3), (2048, 2)]


def _install(C, nbuf, net_classes=0x1F):
    for kb in (4, 8):
        for v in (False, True):
            rc = sn.sn_tuning_set(kb, v, tile_units=C, tile_stages=nbuf, tile_mode=2, net_classes=net_classes)
            if rc != sn.SN_OK:  # a shape too large for this key type: the smallest window instead
                sn.check(sn.sn_tuning_set(kb, v, tile_units=512, tile_stages=2, tile_mode=2,
                                          net_classes=net_classes), "window")


@pytest.fixture(params=WINDOWS, ids=[f"C{c}x{b}" for c, b in WINDOWS])
def window(request):
    _install(*request.param)
    yield request.param
    for kb in (4, 8):
        for v in (False, True):
            sn.check(sn.sn_tuning_set(kb, v), "defaults")


@pytest.mark.parametrize("mode", ["sn", "rss"])
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_window_every_length(window, mode, dtype):
    rng = np.random.default_rng(31)
    lens = np.repeat(np.arange(0, 257, dtype=np.uint32), 4)
    rng.shuffle(lens)
    off = wl.offsets_from_lengths(lens)
    total = int(off[-1])
    for kind in ("uniform", "fewdistinct"):
        k = wl.uniform_keys(total, dtype, seed=32)
        if kind == "fewdistinct":
            k = k % dtype(3)
        v = np.arange(total, dtype=np.uint32)[::-1].copy()
        assert_parity(mode, k, v, off)
        assert_parity(mode, k, None, off)


@pytest.mark.parametrize("mode", ["sn", "rss"])
@pytest.mark.parametrize("lengths,lo,hi", [("uniform", 1, 16), ("geometric", 1, 256), ("uniform", 17, 256)])
def test_window_many_windows(window, mode, lengths, lo, hi):
    k, v, off = wl.segment_batch(1 << 18, lengths, "uniform", np.uint64, True, seed=33, lo=lo, hi=hi)
    assert_parity(mode, k, v, off)
    assert_parity(mode, (k >> np.uint64(40)).astype(np.uint32), None, off)
    kz, _, offz = wl.segment_batch(1 << 16, lengths, "zipf", np.uint32, False, seed=34, lo=lo, hi=hi)
    assert_parity(mode, kz, None, offz)


@pytest.mark.parametrize("net64", [True, False])
def test_window_33_to_64(net64):
    rng = np.random.default_rng(35)
    lens = np.repeat(np.arange(33, 65, dtype=np.uint32), 40)
    rng.shuffle(lens)
    off = wl.offsets_from_lengths(lens)
    total = int(off[-1])
    try:
        _install(1024, 3, net_classes=0x1F if net64 else 0xF)
        for dtype in (np.uint32, np.uint64):
            k = wl.uniform_keys(total, dtype, seed=36)
            k[rng.random(total) < 0.3] = np.iinfo(dtype).max
            k[rng.random(total) < 0.3] = dtype(5)
            v = np.arange(total, dtype=np.uint32)
            assert_parity("sn", k, v, off)
            assert_parity("sn", k, None, off)
    finally:
        for kb in (4, 8):
            for v in (False, True):
                sn.check(sn.sn_tuning_set(kb, v), "defaults")


def test_window_float_keys(window):
    k, v, off = wl.segment_batch(20000, "geometric", "uniform", np.uint32, True, seed=37, p=0.05, cap=256)
    f = (k.view(np.float32)).copy()
    f[::11] = -0.0
    f[::13] = np.float32("nan")
    tk, tv, to_ = to_dev(f.view(np.uint32)), to_dev(v), to_dev(off)
    sn.check(sn.sn_sort_segments_f32(tk, tv, to_), "f32")
    assert sn.sn_check() == sn.SN_OK
    rk, rv = oracle.sort_segments(f, v, off)
    assert np.array_equal(to_host(tk, np.uint32), rk.view(np.uint32))
    assert np.array_equal(to_host(tv, np.uint32), rv)


@pytest.mark.parametrize("mode", ["sn", "rss"])
def test_window_misaligned_pointers(window, mode):
    k, v, off = wl.segment_batch(3000, "geometric", "uniform", np.uint64, True, seed=38)
    for shift in (1, 3):
        pad_k = to_dev(np.concatenate([np.zeros(shift, np.uint64), k]))
        pad_v = to_dev(np.concatenate([np.zeros(shift, np.uint32), v]))
        pad_o = to_dev(np.concatenate([np.zeros(shift, np.uint32), off]))
        fn = sn.sn_sort_segments_u64 if mode == "sn" else sn.rss_sort_segments_u64
        sn.check(fn(pad_k[shift:], pad_v[shift:], pad_o[shift:]), "misaligned")
        sn.check(sn.sn_check())
        rk, rv = oracle.sort_segments(k, v, off)
        assert np.array_equal(to_host(pad_k, np.uint64)[shift:], rk)
        assert np.array_equal(to_host(pad_v, np.uint32)[shift:], rv)
        k32 = (k >> np.uint64(33)).astype(np.uint32)
        pad_k32 = to_dev(np.concatenate([np.zeros(shift, np.uint32), k32]))
        fn32 = sn.sn_sort_segments if mode == "sn" else sn.rss_sort_segments
        sn.check(fn32(pad_k32[shift:], None, pad_o[shift:]), "misaligned u32")
        sn.check(sn.sn_check())
        assert np.array_equal(to_host(pad_k32, np.uint32)[shift:], oracle.sort_segments(k32, None, off)[0])


def test_window_bad_offsets_leave_data_untouched(window):
    for lens_bad in ("long", "decreasing"):
        k, v, off = wl.segment_batch(5000, "uniform", "uniform", np.uint32, True, seed=39)
        off = off.astype(np.int64)
        if lens_bad == "long":
            off[4000:] += 300
        else:
            off[700] = off[699] - 1
        off = off.astype(np.uint32)
        tk, tv, to_ = to_dev(k), to_dev(v), to_dev(off)
        assert sn.sn_sort_segments(tk, tv, to_) == sn.SN_OK
        assert sn.sn_check() == sn.SN_ERANGE
        assert np.array_equal(to_host(tk, np.uint32), k) and np.array_equal(to_host(tv, np.uint32), v)
        assert sn.sn_check() == sn.SN_OK


def test_window_edge_cases(window):
    for dtype in (np.uint32, np.uint64):
        top = np.iinfo(dtype).max
        lens = np.array([0, 1, 256, 0, 2, 33, 17, 16, 256, 1, 0], dtype=np.uint32)
        off = wl.offsets_from_lengths(lens) + np.uint32(5)
        total = int(off[-1]) + 3
        k = wl.uniform_keys(total, dtype, seed=40) % dtype(2)
        k[300:560] = top
        v = np.arange(total, dtype=np.uint32)
        for mode in ("sn", "rss"):
            got_k, got_v = run_segments(mode, k, v, off)
            ref_k, ref_v = oracle.sort_segments(k, v, off)
            assert np.array_equal(got_k, ref_k) and np.array_equal(got_v, ref_v)
        for lens in (np.zeros(1000, np.uint32), np.ones(5000, np.uint32), np.full(3000, 256, np.uint32)):
            off = wl.offsets_from_lengths(lens)
            k = wl.uniform_keys(max(int(off[-1]), 1), dtype, seed=41)
            v = np.arange(k.size, dtype=np.uint32)
            assert_parity("sn", k, v, off)
