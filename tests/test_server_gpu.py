"""The request server: continuous batching over the segmented sort.

Each request's result must be the same when it runs alone and when it is
coalesced with others that arrive while earlier batches are on the GPU:
bit-exact against the oracle's per-segment stable sort either way.  A small
device budget makes admission wait for memory; several slots make batches
overlap.
"""
import threading

import numpy as np
import pytest

import oracle
from paper_2002_05599_gb300 import SN_EINVAL, SN_ERANGE, SN_OK, SmallSortError
from paper_2002_05599_gb300 import workloads as wl
from paper_2002_05599_gb300.server import SortServer, now_ns

pytestmark = pytest.mark.gpu


def _requests(n, dtype, with_vals, seed, max_seg=6000):
    """Mixed requests: segment counts log-uniform in 1..max_seg, lengths 0..256."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        nseg = int(np.exp(rng.uniform(0, np.log(max_seg))))
        dist = ["uniform", "geometric"][i % 2]
        keydist = ["uniform", "fewdistinct"][(i // 2) % 2]
        k, v, off = wl.segment_batch(nseg, dist, keydist, dtype, with_vals, seed=1000 * seed + i, lo=0, hi=256)
        reqs.append((k, v, off))
    return reqs


def _expected(reqs):
    return [oracle.sort_segments(k, v, off) for k, v, off in reqs]


def _run(srv, reqs, threads=1):
    outs = [(np.empty_like(k), None if v is None else np.empty_like(v)) for k, v, _ in reqs]
    tickets = [None] * len(reqs)

    def worker(idx):
        for i in idx:
            k, v, off = reqs[i]
            tickets[i] = srv.submit(k, off, v, outs[i][0], outs[i][1])

    parts = [list(range(t, len(reqs), threads)) for t in range(threads)]
    ths = [threading.Thread(target=worker, args=(p,)) for p in parts]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    for t in tickets:
        assert srv.wait(t) == SN_OK
    return outs


@pytest.mark.parametrize("dtype,with_vals", [(np.uint32, False), (np.uint32, True), (np.uint64, True)])
def test_each_result_same_alone_and_in_the_mix(dtype, with_vals):
    reqs = _requests(24, dtype, with_vals, seed=7 + int(with_vals) + 2 * (dtype == np.uint64))
    expect = _expected(reqs)
    kb = np.dtype(dtype).itemsize
    with SortServer(budget_bytes=48 << 20, key_bytes=kb, slots=3, max_batch_requests=6) as srv:
        alone = []
        for r in reqs:  # one at a time
            alone.append(_run(srv, [r])[0])
        mixed = _run(srv, reqs, threads=4)  # all at once from four client threads
        st = srv.stats()
    for (ek, ev), (ak, av), (mk, mv) in zip(expect, alone, mixed):
        assert np.array_equal(ak, ek) and np.array_equal(mk, ek)
        if with_vals:
            assert np.array_equal(av, ev) and np.array_equal(mv, ev)
    assert st["completed"] == st["submitted"] == 2 * len(reqs)
    assert st["failed"] == 0
    assert st["max_batch_requests_seen"] > 1          # requests were coalesced
    assert st["peak_device_bytes"] <= 48 << 20
    assert 0 < st["latency_p50_us"] <= st["latency_p99_us"] <= st["latency_max_us"]


def test_batches_overlap_and_memory_admission():
    # many mid-size requests, room for only a few at a time
    reqs = _requests(40, np.uint32, False, seed=21, max_seg=20000)
    expect = _expected(reqs)
    with SortServer(budget_bytes=64 << 20, key_bytes=4, slots=4, max_batch_requests=2) as srv:
        out = _run(srv, reqs, threads=2)
        st = srv.stats(reset=True)
        assert srv.stats()["completed"] == 0  # reset cleared the counters
    for (ek, _), (ok, _) in zip(expect, out):
        assert np.array_equal(ok, ek)
    assert st["batches"] >= 20
    assert st["max_inflight_seen"] >= 2  # batches were on the GPU at the same time
    assert st["peak_device_bytes"] <= 64 << 20


def test_in_place_and_offsets_not_starting_at_zero():
    k, v, off = wl.segment_batch(3000, "uniform", "uniform", np.uint32, True, seed=5, lo=0, hi=256)
    ek, ev = oracle.sort_segments(k, v, off)
    # the request covers segments 1000..2999 only, addressed in the full arrays
    sub = off[1000:].copy()
    kk, vv = k.copy(), v.copy()
    with SortServer(budget_bytes=32 << 20) as srv:
        t = srv.submit(kk, sub, vv)  # in place
        assert srv.wait(t) == SN_OK
    lo = int(off[1000])
    assert np.array_equal(kk[:lo], k[:lo]) and np.array_equal(vv[:lo], v[:lo])  # untouched
    assert np.array_equal(kk[lo:], ek[lo:]) and np.array_equal(vv[lo:], ev[lo:])


def test_rejections_and_empty_requests():
    with SortServer(budget_bytes=1 << 20, key_bytes=4) as srv:
        k = np.zeros(1 << 20, np.uint32)  # 4 MB of keys: more than the whole budget
        off = np.arange(0, (1 << 20) + 1, 256, dtype=np.uint32)
        with pytest.raises(SmallSortError) as e:
            srv.submit(k, off)
        assert e.value.status == SN_ERANGE
        bad = np.array([0, 5, 3], np.uint32)  # decreasing
        with pytest.raises(SmallSortError) as e:
            srv.submit(np.zeros(8, np.uint32), bad)
        assert e.value.status == SN_ERANGE
        long_seg = np.array([0, 257], np.uint32)  # longer than 256
        with pytest.raises(SmallSortError) as e:
            srv.submit(np.zeros(257, np.uint32), long_seg)
        assert e.value.status == SN_ERANGE
        t = srv.submit(np.zeros(0, np.uint32), np.zeros(1, np.uint32))  # no segments
        assert srv.wait(t, 0) == SN_OK
        assert srv.wait(t, 0) == SN_EINVAL  # already collected
        assert srv.wait(123456789, 0) == SN_EINVAL


def test_arrival_times_enter_the_latency():
    k, v, off = wl.segment_batch(2000, "uniform", "uniform", np.uint32, False, seed=9, lo=2, hi=256)
    with SortServer(budget_bytes=32 << 20) as srv:
        t = srv.submit(k.copy(), off, arrival_ns=now_ns() - 50_000_000)  # arrived 50 ms ago
        assert srv.wait(t) == SN_OK
        st = srv.stats()
    assert st["latency_p50_us"] >= 50_000
