"""The multi-GPU path of the benchmark is replicas (every rank sorts its own
batch, no data exchange): its host-side logic -- per-rank inputs, the
max-over-ranks timing, the whole-job throughput -- checked with two gloo
ranks on the CPU, each rank sorting its batch with the CPU oracle."""
import os
import socket

import numpy as np
import pytest

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = bench.workload_sizes(14)  # a tiny version of every workload
        inp = bench.make_inputs(sizes, "cpu", rank, parts=("sweep", "uneven", "rss"))
        # each rank sorts its own batch (here with the oracle) and times it
        keys = inp["rss_keys"].numpy().view(np.uint32)
        off = inp["rss_off"].numpy().view(np.uint32)
        got, _ = oracle.sort_segments(keys, None, off)
        ok = bool(oracle.is_sorted_segments(got, off))
        my_times = [1.0 + rank, 5.0 - rank]
        reduced = bench.max_over_ranks(my_times, dist, "cpu")
        job_keys = bench.sum_over_ranks([keys.size], dist, "cpu")[0]
        out.put((rank, ok, reduced, int(keys[:8].sum()), inp["rss_off"].numel(),
                 bench.job_throughput(job_keys, reduced[0]), keys.size, job_keys))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ok0, red0, sig0, nseg0, thr0, k0, job0), (r1, ok1, red1, sig1, nseg1, thr1, k1, job1) = res
    assert ok0 and ok1
    assert red0 == red1 == [2.0, 5.0]          # element-wise maximum over the ranks
    assert sig0 != sig1 and nseg0 == nseg1     # own inputs per rank, same number of segments
    assert job0 == job1 == k0 + k1             # every rank's keys count (their lengths differ)
    assert thr0 == thr1 == (k0 + k1) / 2.0     # the same job throughput on every rank


def test_single_process_reduction_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 1.0], None, "cpu") == [3.0, 1.0]
    assert bench.sum_over_ranks([7.0], None, "cpu") == [7.0]
    assert bench.job_throughput(400, 2.0) == 200.0
