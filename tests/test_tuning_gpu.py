"""Launch parameters change speed only: every parameter set sorts a batch to
the oracle's result, and the autotuner leaves the batch sorted and installs
the set it reports."""
import numpy as np
import pytest

import oracle
import paper_2002_05599_gb300 as sn
from paper_2002_05599_gb300 import workloads as wl
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

SETS = [dict(tile_units=512, net_classes=0x0, rss_two_min=16, tile_stages=2, tile_mode=0),
        dict(tile_units=4096, net_classes=0xF, rss_two_min=256, tile_stages=2, tile_mode=1),
        dict(tile_units=1024, net_classes=0x15, rss_two_min=64, tile_stages=4, tile_mode=0),
        dict(tile_units=2048, net_classes=0xA, rss_two_min=200, tile_stages=3, tile_mode=1),
        dict(tile_units=512, net_classes=0x14, rss_two_min=128, tile_stages=3, tile_mode=1),
        dict(tile_units=1024, net_classes=0x0, rss_two_min=160, tile_stages=4, tile_mode=1),
        # tile sizes that are neither a power of two nor 3 * 2^k: the plan
        # kernel's general tile division (and 3 * 2^k, its multiply-high path)
        dict(tile_units=1000, net_classes=0x1F, rss_two_min=160, tile_stages=2, tile_mode=0),
        dict(tile_units=1537, net_classes=0x1F, rss_two_min=160, tile_stages=2, tile_mode=1),
        dict(tile_units=1536, net_classes=0x1F, rss_two_min=160, tile_stages=2, tile_mode=0)]


@pytest.fixture
def restore_defaults():
    yield
    for kb in (4, 8):
        for v in (False, True):
            sn.check(sn.sn_tuning_set(kb, v), "defaults")


@pytest.mark.parametrize("dtype,with_vals", [(np.uint64, True), (np.uint32, False), (np.uint32, True)])
def test_every_parameter_set_gives_the_same_result(dtype, with_vals, restore_defaults):
    kb = np.dtype(dtype).itemsize
    fn = sn.sn_sort_segments_u64 if kb == 8 else sn.sn_sort_segments
    rss = sn.rss_sort_segments_u64 if kb == 8 else sn.rss_sort_segments
    k, v, off = wl.segment_batch(60_000, "uniform", "fewdistinct", dtype, with_vals, seed=77, lo=0, hi=256)
    ek, ev = oracle.sort_segments(k, v, off)
    d_off = to_dev(off)
    for params in SETS:
        sn.check(sn.sn_tuning_set(kb, with_vals, **params), "set")
        assert sn.sn_tuning_get(kb, with_vals) == params
        for call in (fn, rss):
            dk = to_dev(k)
            dv = to_dev(v) if with_vals else None
            sn.check(call(dk, dv, d_off), "sort")
            assert sn.sn_check() == sn.SN_OK
            assert np.array_equal(to_host(dk, dtype), ek), params
            if with_vals:
                assert np.array_equal(to_host(dv, np.uint32), ev), params


def test_tile_size_limit_by_shared_memory(restore_defaults):
    # ring kernel (packed stages): a stage takes max(6, key + payload bytes) per
    # unit of tile_units + 256, and a block at most 223 KB
    assert sn.sn_tuning_set(4, False, tile_units=8192, tile_stages=4) == sn.SN_OK   # 6 B per unit
    assert sn.sn_tuning_set(4, False, tile_units=16384, tile_stages=2) == sn.SN_OK
    assert sn.sn_tuning_set(4, False, tile_units=16384, tile_stages=3) == sn.SN_EINVAL
    for kb, v in ((4, True), (8, False)):                                           # 8 B per unit
        assert sn.sn_tuning_set(kb, v, tile_units=8192, tile_stages=3) == sn.SN_OK
        assert sn.sn_tuning_set(kb, v, tile_units=8192, tile_stages=4) == sn.SN_EINVAL
    assert sn.sn_tuning_set(8, True, tile_units=8192, tile_stages=2) == sn.SN_OK    # 12 B per unit
    assert sn.sn_tuning_set(8, True, tile_units=8192, tile_stages=3) == sn.SN_EINVAL
    assert sn.sn_tuning_set(8, True, tile_units=4096, tile_stages=4) == sn.SN_OK
    # synchronous kernel (fixed regions): two 8192-unit stages only for u32 keys alone
    assert sn.sn_tuning_set(4, False, tile_units=8192, tile_mode=1) == sn.SN_OK
    for kb, v in ((4, True), (8, False), (8, True)):
        assert sn.sn_tuning_set(kb, v, tile_units=8192, tile_mode=1) == sn.SN_EINVAL
    # the largest shapes sort correctly
    k, _, off = wl.segment_batch(50_000, "geometric", "uniform", np.uint32, False, seed=79, p=0.15, cap=256)
    dk = to_dev(k)
    for units, stages in ((8192, 4), (16384, 2)):
        dk = to_dev(k)
        sn.check(sn.sn_tuning_set(4, False, tile_units=units, tile_stages=stages), "set")
        sn.check(sn.sn_sort_segments(dk, None, to_dev(off)), "sort")
        assert sn.sn_check() == sn.SN_OK
        assert np.array_equal(to_host(dk, np.uint32), oracle.sort_segments(k, None, off)[0]), units
    k, v, off = wl.segment_batch(60_000, "geometric", "fewdistinct", np.uint64, True, seed=80, p=0.15, cap=256)
    ek, ev = oracle.sort_segments(k, v, off)
    for units, stages in ((8192, 2), (6144, 2), (4096, 4), (3072, 3)):
        dk, dv = to_dev(k), to_dev(v)
        sn.check(sn.sn_tuning_set(8, True, tile_units=units, tile_stages=stages), "set")
        sn.check(sn.sn_sort_segments_u64(dk, dv, to_dev(off)), "sort")
        assert sn.sn_check() == sn.SN_OK
        assert np.array_equal(to_host(dk, np.uint64), ek) and np.array_equal(to_host(dv, np.uint32), ev), units


def test_autotuner_installs_its_choice_and_sorts(tmp_path, restore_defaults):
    k, v, off = wl.segment_batch(1 << 18, "geometric", "uniform", np.uint64, True, seed=78, p=0.15, cap=256)
    ek, ev = oracle.sort_segments(k, v, off)
    dk, dv, d_off = to_dev(k), to_dev(v), to_dev(off)
    params, ms = sn.sn_tune_segments(dk, dv, d_off)
    assert ms > 0
    assert sn.sn_tuning_get(8, True) == params
    assert np.array_equal(to_host(dk, np.uint64), ek) and np.array_equal(to_host(dv, np.uint32), ev)
    path = str(tmp_path / "tuning.txt")
    assert sn.sn_tuning_save(path) == sn.SN_OK
    sn.check(sn.sn_tuning_set(8, True), "reset")
    assert sn.sn_tuning_load(path) == sn.SN_OK
    assert sn.sn_tuning_get(8, True) == params


def test_rss_autotuner_times_the_rss_call(restore_defaults):
    # the RSS-mode search leaves a batch sorted by rss_sort_segments, with
    # every segment over 16 items through Register Sample Sort
    k, _, off = wl.segment_batch(1 << 16, "uniform", "zipf", np.uint32, False, seed=81, lo=17, hi=256)
    ek = oracle.sort_segments(k, None, off)[0]
    dk, d_off = to_dev(k), to_dev(off)
    params, ms = sn.sn_tune_segments(dk, None, d_off, rss_only=True)
    # the tile kernel with the RSS kernel (mode 0) or the one-launch window kernel (mode 2)
    assert ms > 0 and params["tile_mode"] in (0, 2)
    assert sn.sn_tuning_get(4, False) == params
    assert np.array_equal(to_host(dk, np.uint32), ek)


@pytest.mark.parametrize("dtype,with_vals", [(np.uint64, True), (np.uint32, False), (np.uint32, True), (np.uint64, False)])
@pytest.mark.parametrize("lengths,lo,hi", [("geometric", 1, 256), ("uniform", 0, 40)])
def test_synchronous_tile_mode_many_tiles(dtype, with_vals, lengths, lo, hi, restore_defaults):
    # the synchronous tile kernel over enough tiles that every block reuses its stages
    kb = np.dtype(dtype).itemsize
    fn = sn.sn_sort_segments_u64 if kb == 8 else sn.sn_sort_segments
    for stages, units in ((2, 2048), (3, 1024), (4, 512)):
        sn.check(sn.sn_tuning_set(kb, with_vals, tile_units=units, tile_stages=stages, tile_mode=1), "set")
        for keys in ("uniform", "fewdistinct"):
            k, v, off = wl.segment_batch(1 << 17, lengths, keys, dtype, with_vals, seed=80 + stages, lo=lo, hi=hi)
            ek, ev = oracle.sort_segments(k, v, off)
            dk, dv = to_dev(k), (to_dev(v) if with_vals else None)
            sn.check(fn(dk, dv, to_dev(off)), "sort")
            assert sn.sn_check() == sn.SN_OK
            assert np.array_equal(to_host(dk, dtype), ek)
            if with_vals:
                assert np.array_equal(to_host(dv, np.uint32), ev)


def test_sn_tune_tunes_saves_and_loads(tmp_path, restore_defaults):
    # sn_tune(path): with no file, tunes the four key type / payload kinds on
    # the library's synthetic batch, installs them and writes the file; with
    # the file, loads it.  The sets it chose sort like any other.
    path = str(tmp_path / "tuned.txt")
    assert sn.sn_tune(path) == sn.SN_OK
    chosen = {(kb, v): sn.sn_tuning_get(kb, v) for kb in (4, 8) for v in (False, True)}
    assert open(path).read().startswith("smallsort-tuning")
    for kb in (4, 8):
        for v in (False, True):
            sn.check(sn.sn_tuning_set(kb, v), "reset")
    assert sn.sn_tune(path) == sn.SN_OK  # the file now exists: a load
    assert {(kb, v): sn.sn_tuning_get(kb, v) for kb in (4, 8) for v in (False, True)} == chosen
    k, v, off = wl.segment_batch(40_000, "geometric", "fewdistinct", np.uint64, True, seed=82, p=0.15, cap=256)
    ek, ev = oracle.sort_segments(k, v, off)
    dk, dv = to_dev(k), to_dev(v)
    sn.check(sn.sn_sort_segments_u64(dk, dv, to_dev(off)), "sort")
    assert sn.sn_get_last_cuda_error() == sn.SN_OK
    assert np.array_equal(to_host(dk, np.uint64), ek) and np.array_equal(to_host(dv, np.uint32), ev)
    bad = tmp_path / "bad.txt"
    bad.write_text("not a tuning file\n")
    assert sn.sn_tune(str(bad)) == sn.SN_EINVAL
