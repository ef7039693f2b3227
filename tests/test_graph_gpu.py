"""The segmented sort captured in a CUDA graph and replayed on new data.

Under stream capture the call records its scratch as a graph allocation node,
so the graph is self-contained: replays on fresh keys with the same offsets
must match the oracle exactly, like direct calls."""
import numpy as np
import pytest

import oracle
import paper_2002_05599_gb300 as sn
from paper_2002_05599_gb300 import workloads as wl
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,with_vals,lengths", [(np.uint64, True, "geometric"), (np.uint32, False, "uniform")])
def test_segmented_sort_replays_from_a_captured_graph(dtype, with_vals, lengths):
    import torch
    fn = sn.sn_sort_segments_u64 if dtype == np.uint64 else sn.sn_sort_segments
    nseg = 200_000
    hi = 256 if lengths == "uniform" else 16
    k0, v0, off = wl.segment_batch(nseg, lengths, "uniform", dtype, with_vals, seed=41, lo=1, hi=hi)
    keys, d_off = to_dev(k0), to_dev(off)
    vals = to_dev(v0) if with_vals else None
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):  # first call outside capture: device set-up
        sn.check(fn(keys, vals, d_off), "warm-up")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        rc = fn(keys, vals, d_off)
    assert rc == sn.SN_OK
    for seed in (42, 43):
        kk = wl.uniform_keys(k0.size, dtype, seed)
        keys.copy_(to_dev(kk))
        if with_vals:
            vals.copy_(to_dev(v0))
        graph.replay()
        torch.cuda.synchronize()
        assert sn.sn_check() == sn.SN_OK
        ek, ev = oracle.sort_segments(kk, v0 if with_vals else None, off)
        assert np.array_equal(to_host(keys, dtype), ek)
        if with_vals:
            assert np.array_equal(to_host(vals, np.uint32), ev)
