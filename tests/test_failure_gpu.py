"""Failure detection on the GPU without a fault.

Every wait inside the library's kernels is bounded.  A test flag
(include/smallsort_testing.h) makes one kernel arm its copy-completion
barrier without issuing the copy, so that kernel's own wait, shortened here to
a few milliseconds, runs out: the kernel records SN_ETIMEOUT in the status
word and returns.  Nothing traps, nothing spins without a limit, and the
device stays usable: the same call without the flag then sorts to the
oracle's result.  The request server reports such a batch's failure on its
requests (a status word per batch), and later requests complete normally.
"""
import ctypes
import threading
import time

import numpy as np
import pytest

import oracle
import paper_2002_05599_gb300 as sn
from paper_2002_05599_gb300 import workloads as wl
from paper_2002_05599_gb300.server import SortServer
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

SKIP_FIXED, SKIP_TILE, SKIP_RSS = 1, 2, 4  # SN_TEST_SKIP_* in include/smallsort_testing.h
LIMIT_NS = 5_000_000  # 5 ms


def _hooks():
    lib = sn.library()
    lib.sn_test_set_flags.argtypes = [ctypes.c_uint]
    lib.sn_test_set_flags.restype = ctypes.c_int
    lib.sn_set_wait_limit.argtypes = [ctypes.c_uint64]
    lib.sn_set_wait_limit.restype = ctypes.c_int
    return lib


@pytest.fixture
def hooks():
    lib = _hooks()
    assert lib.sn_set_wait_limit(LIMIT_NS) == sn.SN_OK
    yield lib
    assert lib.sn_test_set_flags(0) == sn.SN_OK
    assert lib.sn_set_wait_limit(2_000_000_000) == sn.SN_OK
    assert sn.sn_check() == sn.SN_OK


def test_hook_arguments():
    lib = _hooks()
    assert lib.sn_set_wait_limit(999) == sn.SN_EINVAL
    assert lib.sn_set_wait_limit(60_000_000_001) == sn.SN_EINVAL
    assert lib.sn_test_set_flags(8) == sn.SN_EINVAL


def _timed_out(call):
    t0 = time.perf_counter()
    assert call() == sn.SN_OK  # the launch itself succeeds; the failure is found on the device
    status = sn.sn_check()
    return status, time.perf_counter() - t0


def test_fixed_kernel_wait_runs_out_and_device_recovers(hooks):
    keys = wl.fixed_arrays(8, 1 << 18, "uniform", np.uint32, seed=41)
    t = to_dev(keys)
    assert hooks.sn_test_set_flags(SKIP_FIXED) == sn.SN_OK
    status, secs = _timed_out(lambda: sn.sn_sort_fixed(t, 8))
    assert status == sn.SN_ETIMEOUT
    assert secs < 5.0  # a few bounded waits of 5 ms, not the 2 s default
    assert hooks.sn_test_set_flags(0) == sn.SN_OK
    t = to_dev(keys)
    sn.check(sn.sn_sort_fixed(t, 8), "sort")
    assert sn.sn_check() == sn.SN_OK
    assert np.array_equal(to_host(t, np.uint32), oracle.sort_fixed(keys, 8))


@pytest.mark.parametrize("flag,lo,hi,call", [(SKIP_TILE, 1, 32, "sn"), (SKIP_RSS, 17, 256, "rss")])
def test_segmented_kernel_wait_runs_out_and_device_recovers(hooks, flag, lo, hi, call):
    fn = sn.sn_sort_segments_u64 if call == "sn" else sn.rss_sort_segments_u64
    k, v, off = wl.segment_batch(1 << 15, "uniform", "uniform", np.uint64, True, seed=42, lo=lo, hi=hi)
    dk, dv, doff = to_dev(k), to_dev(v), to_dev(off)
    assert hooks.sn_test_set_flags(flag) == sn.SN_OK
    status, secs = _timed_out(lambda: fn(dk, dv, doff))
    assert status == sn.SN_ETIMEOUT
    assert secs < 5.0
    # the device-wide form reports the same kind of failure
    assert fn(dk, dv, doff) == sn.SN_OK
    assert sn.sn_get_last_cuda_error() == sn.SN_ETIMEOUT
    assert hooks.sn_test_set_flags(0) == sn.SN_OK
    dk, dv = to_dev(k), to_dev(v)
    sn.check(fn(dk, dv, doff), "sort")
    assert sn.sn_check() == sn.SN_OK
    ek, ev = oracle.sort_segments(k, v, off)
    assert np.array_equal(to_host(dk, np.uint64), ek) and np.array_equal(to_host(dv, np.uint32), ev)


def test_server_request_reports_its_batch_failure(hooks):
    k, v, off = wl.segment_batch(5000, "uniform", "uniform", np.uint32, True, seed=43, lo=0, hi=256)
    ek, ev = oracle.sort_segments(k, v, off)
    with SortServer(1 << 28, key_bytes=4, slots=2) as srv:
        assert hooks.sn_test_set_flags(SKIP_TILE | SKIP_RSS) == sn.SN_OK
        ok, ov = np.empty_like(k), np.empty_like(v)
        t = srv.submit(k, off, v, ok, ov)
        assert srv.wait(t) == sn.SN_ECUDA  # a bounded device wait of its batch ran out
        assert srv.stats()["failed"] == 1
        assert hooks.sn_test_set_flags(0) == sn.SN_OK
        ok, ov = np.empty_like(k), np.empty_like(v)
        t = srv.submit(k, off, v, ok, ov)
        assert srv.wait(t) == sn.SN_OK
        assert np.array_equal(ok, ek) and np.array_equal(ov, ev)
    # the server's kernels report into their batch's word, not the device's
    assert sn.sn_check() == sn.SN_OK


def test_two_threads_waiting_on_one_ticket():
    k, v, off = wl.segment_batch(20000, "uniform", "uniform", np.uint32, True, seed=44, lo=0, hi=256)
    with SortServer(1 << 28, key_bytes=4, slots=2) as srv:
        ok, ov = np.empty_like(k), np.empty_like(v)
        t = srv.submit(k, off, v, ok, ov)
        got = []
        ths = [threading.Thread(target=lambda: got.append(srv.wait(t))) for _ in range(2)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        assert sorted(got) == sorted([sn.SN_OK, sn.SN_EINVAL])  # one collects it, the other finds it gone
        assert srv.wait(t) == sn.SN_EINVAL
