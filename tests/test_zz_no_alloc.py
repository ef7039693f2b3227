"""The allocation-free segmented sort against the allocating one.

sn_sort_segments_u64_noalloc exists for callers that cannot allocate device
memory when they sort (a fixed budget reserved up front, a thread that must
not enter the allocator).  Its scratch is a fixed array inside the library
that every call reuses, so this test runs it twice in a row on different
batches and checks each result bit for bit against sn_sort_segments_u64 on a
copy of the same input, and against the CPU oracle's per-segment stable sort.
It also checks the size limit.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2002_05599_gb300 as sn
from paper_2002_05599_gb300 import workloads as wl
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

MAX_SEGMENTS = 262144  # SN_NOALLOC_MAX_SEGMENTS in include/smallsort.h


def _lib():
    lib = sn.library()
    fn = lib.sn_sort_segments_u64_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return lib


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    lib = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    batches = [
        wl.segment_batch(MAX_SEGMENTS, "geometric", "uniform", np.uint64, True, seed=31),
        wl.segment_batch(50000, "uniform", "fewdistinct", np.uint64, True, seed=32, lo=1, hi=256),
    ]
    for k, v, off in batches:  # two calls in a row share the library's scratch
        ref_k, ref_v = to_dev(k), to_dev(v)
        got_k, got_v = to_dev(k), to_dev(v)
        d_off = to_dev(off)
        nseg = off.size - 1
        assert lib.sn_sort_segments_u64(ref_k.data_ptr(), ref_v.data_ptr(), d_off.data_ptr(), nseg, stream) == 0
        assert lib.sn_sort_segments_u64_noalloc(got_k.data_ptr(), got_v.data_ptr(), d_off.data_ptr(), nseg,
                                                stream) == 0
        assert sn.sn_check() == sn.SN_OK
        assert np.array_equal(to_host(got_k, np.uint64), to_host(ref_k, np.uint64))
        assert np.array_equal(to_host(got_v, np.uint32), to_host(ref_v, np.uint32))
        ek, ev = oracle.sort_segments(k, v, off)  # element by element against the oracle
        assert np.array_equal(to_host(got_k, np.uint64), ek)
        assert np.array_equal(to_host(got_v, np.uint32), ev)
        # keys only
        got_k2 = to_dev(k)
        assert lib.sn_sort_segments_u64_noalloc(got_k2.data_ptr(), None, d_off.data_ptr(), nseg, stream) == 0
        assert sn.sn_check() == sn.SN_OK
        assert np.array_equal(to_host(got_k2, np.uint64), to_host(ref_k, np.uint64))


def test_noalloc_rejects_batches_above_its_limit():
    lib = _lib()
    k, v, off = wl.segment_batch(MAX_SEGMENTS + 1, "uniform", "uniform", np.uint64, True, seed=33)
    dk, dv, doff = to_dev(k), to_dev(v), to_dev(off)
    rc = lib.sn_sort_segments_u64_noalloc(dk.data_ptr(), dv.data_ptr(), doff.data_ptr(), MAX_SEGMENTS + 1, None)
    assert rc == sn.SN_ERANGE
    assert np.array_equal(to_host(dk, np.uint64), k)  # nothing was launched
