#!/usr/bin/env python
"""Benchmark of batched small-set sorting on GB300 (one JSON line on stdout).

One step sorts one batch of every workload of the hot path, device-resident:
  * sweep   -- fixed n = 2..16: 2^24 arrays per n of uniform u32 keys
               (sn_sort_fixed, one launch per n);
  * uneven  -- 2^24 CSR segments, lengths geometric(p = 0.15) capped at 256,
               uniform u64 keys with a u32 payload = original index
               (sn_sort_segments_u64: plan + one persistent launch);
  * rss     -- 2^20 segments of 17..256 uniform u32 keys, keys only
               (rss_sort_segments: plan + one persistent launch).
Before every step (outside the timed window) the work buffers are restored
from pristine copies, which also evicts L2 (the step touches ~12 GB, L2 is
126 MB).  Each step is timed with CUDA events on the launching stream.

value     = sorted keys of all parts and ranks / step time (Gkeys/s).
roofline  = the fixed-n network kernel (sweep): algorithmic bytes (8 B per u32
            key: read + write) over its measured time, against the measured
            HBM copy bandwidth.
e2e       = the same step through the C ABI with host buffers: pinned
            host -> device copies of the inputs, the sorts, device -> host
            copies of the results, all inside the timed region.
cpu_baseline / --impl reference = the CPU oracle (insertion sort, one core)
            on a bounded sample of the same workload.

Multi-GPU (torchrun): every rank sorts its own full batch (replicas, weak
scaling); no data-path collective.  Timing: barrier + synchronize around the
K timed steps, maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SWEEP_NS = list(range(2, 17))
# DRAM bytes (read + write) of one full-size sweep step, from an ncu capture of the
# fixed-n kernel at 2^22 arrays per n scaled to 2^24 (reads equal the algorithmic
# reads; writes fall short by the output still resident in L2 at each kernel's end).
SWEEP_DRAM_BYTES = 17_216_000_000
FALLBACK_HBM_GBS = 6800.0
METRIC = "sorted Gkeys/s at 1 GB300 and % of HBM roofline"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=int, default=0,
                    help="divide every workload by 2^scale (debugging only; default full size)")
    ap.add_argument("--parts", default="sweep,uneven,rss",
                    help="comma-separated subset of sweep,uneven,rss (profiling only; default all)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="call the uneven batch directly instead of replaying its captured CUDA graph")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-vs-batched comparison")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch parameters instead of autotuning each segmented workload")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving loop")
    ap.add_argument("--tuning", default="",
                    help="parameter file: loaded if it exists (no autotuning), else written after autotuning, "
                         "so that a profiled run uses the timed run's launch parameters")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip config 1 (cold L2), config 2's other distributions and config 3 (i)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the float-key and long-segment measurements")
    ap.add_argument("--no-families", action="store_true",
                    help="skip the network-family comparison (best known vs Bose-Nelson, u32 keys and 16-byte items)")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="length of the Poisson request stream")
    ap.add_argument("--serve-rate", type=float, default=20000.0, help="mean request arrival rate (1/s)")
    return ap.parse_args()


def workload_sizes(scale: int):
    return {"sweep_count": (1 << 24) >> scale, "uneven_nseg": (1 << 24) >> scale,
            "rss_nseg": (1 << 20) >> scale}


def config_dict(sizes, scale):
    wl = ("fixed-n sweep n=2..16 x 2^24 arrays u32 uniform + uneven batch 2^24 segments "
          "geometric(0.15) cap 256 u64 keys + u32 payload + RSS range 2^20 segments 17..256 u32 uniform")
    if scale:
        wl += f" (all sizes / 2^{scale})"
    return {"workload": wl, "sweep_arrays_per_n": sizes["sweep_count"],
            "uneven_segments": sizes["uneven_nseg"], "rss_segments": sizes["rss_nseg"],
            "seed": 1, "l2": "inputs larger than L2; buffers restored from pristine copies between steps, "
                             "then the sweep (about 18 GB of traffic) runs before the uneven and RSS parts, so "
                             "no part's input is still in L2 from the restore",
            "parallelism": "replicas (one independent batch per GPU)"}


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings over all ranks (identity without
    a process group): the job's time is its slowest rank's."""
    if not dist:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def sum_over_ranks(values, dist, device):
    """Element-wise sum over all ranks (identity without a process group)."""
    if not dist:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.tolist()


def job_throughput(units_all_ranks, seconds):
    """Whole-job throughput of weakly scaled replicas: the units every rank
    processed, summed over the ranks, divided by the slowest rank's time."""
    return units_all_ranks / seconds


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for name, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- our arm ----

def make_inputs(sizes, device, rank, parts=("sweep", "uneven", "rss")):
    import torch
    from paper_2002_05599_gb300 import workloads as wl
    seed = 1 + rank
    inp = {}
    if "sweep" in parts:
        for n in SWEEP_NS:
            inp[f"sweep{n}"] = wl.uniform_keys_torch(sizes["sweep_count"] * n, np.uint32, seed=seed * 1000 + n,
                                                     device=device)
    if "uneven" in parts:
        lens = wl.segment_lengths(sizes["uneven_nseg"], "geometric", seed=seed, p=0.15, cap=256)
        off = wl.offsets_from_lengths(lens)
        total = int(off[-1])
        inp["uneven_off"] = torch.from_numpy(off.view(np.int32)).to(device)
        inp["uneven_keys"] = wl.uniform_keys_torch(total, np.uint64, seed=seed, device=device)
        inp["uneven_vals"] = torch.arange(total, dtype=torch.int32, device=device)
    if "rss" in parts:
        lens = wl.segment_lengths(sizes["rss_nseg"], "uniform", seed=seed + 100, lo=17, hi=256)
        off = wl.offsets_from_lengths(lens)
        inp["rss_off"] = torch.from_numpy(off.view(np.int32)).to(device)
        inp["rss_keys"] = wl.uniform_keys_torch(int(off[-1]), np.uint32, seed=seed + 100, device=device)
    return inp


def part_keys(inp):
    out = {}
    if "sweep2" in inp:
        out["sweep"] = sum(inp[f"sweep{n}"].numel() for n in SWEEP_NS)
    if "uneven_keys" in inp:
        out["uneven"] = inp["uneven_keys"].numel()
    if "rss_keys" in inp:
        out["rss"] = inp["rss_keys"].numel()
    return out


def part_bytes(inp):
    """Algorithmic bytes per step: every key / payload read and written once,
    offsets read once."""
    out = {}
    if "sweep2" in inp:
        out["sweep"] = 8 * sum(inp[f"sweep{n}"].numel() for n in SWEEP_NS)
    if "uneven_keys" in inp:
        out["uneven"] = 2 * (8 + 4) * inp["uneven_keys"].numel() + 4 * inp["uneven_off"].numel()
    if "rss_keys" in inp:
        out["rss"] = 2 * 4 * inp["rss_keys"].numel() + 4 * inp["rss_off"].numel()
    return out


def launches_per_step(parts=("sweep", "uneven", "rss")):
    """Kernels of this library launched per step: one per fixed n, and plan,
    bin, tile and RSS kernels per segmented call."""
    return (len(SWEEP_NS) if "sweep" in parts else 0) + 4 * sum(p in parts for p in ("uneven", "rss"))


PARTS = ("sweep", "uneven", "rss")


def run_parts(sn, w, events=None, parts=PARTS, graphs=None, n_events=None):
    """One step on the current stream; events[0..3] bracket sweep / uneven / rss,
    n_events[i] (optional) follows the sort of the i-th fixed n.
    graphs["uneven"], when given, is the captured uneven-batch call."""
    if events:
        events[0].record()
    if "sweep" in parts:
        for i, n in enumerate(SWEEP_NS):
            sn.check(sn.sn_sort_fixed(w[f"sweep{n}"], n), f"sn_sort_fixed n={n}")
            if n_events:
                n_events[i].record()
    if events:
        events[1].record()
    if "uneven" in parts:
        if graphs and "uneven" in graphs:
            graphs["uneven"].replay()
        else:
            sn.check(sn.sn_sort_segments_u64(w["uneven_keys"], w["uneven_vals"], w["uneven_off"]), "uneven")
    if events:
        events[2].record()
    if "rss" in parts:
        sn.check(sn.rss_sort_segments(w["rss_keys"], None, w["rss_off"]), "rss")
    if events:
        events[3].record()


def bench_ours(args, rank, world, local_rank, dist):
    import torch
    import paper_2002_05599_gb300 as sn

    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    sizes = workload_sizes(args.scale)
    parts = tuple(p for p in args.parts.split(",") if p)
    pristine = make_inputs(sizes, device, rank, parts)
    work = {k: v.clone() for k, v in pristine.items()}
    keys = part_keys(pristine)
    bytes_ = part_bytes(pristine)
    total_keys = sum(keys.values())

    def restore():
        for k, v in work.items():
            if not k.endswith("_off"):
                v.copy_(pristine[k])

    for _ in range(args.warmup):
        restore()
        run_parts(sn, work, parts=parts)
    torch.cuda.synchronize()
    status = sn.sn_check()
    sn.check(status, "warm-up")
    tuned = {}
    if args.tuning and os.path.exists(args.tuning):  # the parameters a previous run tuned and saved
        sn.check(sn.sn_tuning_load(args.tuning), "sn_tuning_load")
        tuned = {"loaded": args.tuning,
                 "uneven": sn.sn_tuning_get(8, True), "rss": sn.sn_tuning_get(4, False)}
    elif not args.no_tune:  # autotune each segmented workload on its own batch (untimed)
        restore()  # on unsorted input: the warm-up left the batches sorted
        if "uneven" in parts:
            tuned["uneven"] = autotune(sn, work["uneven_keys"], work["uneven_vals"], work["uneven_off"])
        if "rss" in parts:
            tuned["rss"] = autotune(sn, work["rss_keys"], None, work["rss_off"], rss_only=True)
        if args.tuning:
            sn.check(sn.sn_tuning_save(args.tuning), "sn_tuning_save")
    graphs = {}
    if "uneven" in parts and not args.no_graph:
        graphs["uneven"] = capture_uneven(sn, work)
        restore()
        run_parts(sn, work, parts=("uneven",), graphs=graphs)
        torch.cuda.synchronize()
        sn.check(sn.sn_check(), "graph warm-up")

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    nev = [[torch.cuda.Event(enable_timing=True) for _ in SWEEP_NS] for _ in range(args.steps)]
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    t0 = time.perf_counter()
    for k in range(args.steps):
        restore()
        run_parts(sn, work, ev[k], parts=parts, graphs=graphs, n_events=nev[k])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = sampler.stop() if sampler else None
    if dist:
        dist.barrier()
    sn.check(sn.sn_check(), "timed steps")

    per = {"sweep": [], "uneven": [], "rss": [], "step": []}
    for e in ev:
        a, b, c, d = (e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3]),
                      e[0].elapsed_time(e[3]))
        per["sweep"].append(a)
        per["uneven"].append(b)
        per["rss"].append(c)
        per["step"].append(d)
    ms = {k: statistics.mean(v) for k, v in per.items()}
    ms = dict(zip(["step", "sweep", "uneven", "rss"],
                  max_over_ranks([ms["step"], ms["sweep"], ms["uneven"], ms["rss"]], dist, device)))

    hbm, hbm_src = peaks()
    sweep_gbs = bytes_["sweep"] / (ms["sweep"] * 1e-3) / 1e9 if "sweep" in parts else 0.0
    parts_out = {}
    if "sweep" in parts:  # per n: time between the events around its launch, mean over steps
        per_n = {}
        for i, n in enumerate(SWEEP_NS):
            t = statistics.mean((e[0] if i == 0 else ne[i - 1]).elapsed_time(ne[i]) for e, ne in zip(ev, nev))
            b = 8 * pristine[f"sweep{n}"].numel()
            per_n[n] = {"ms": round(t, 4), "gkeys_s": round(b / 8 / (t * 1e-3) / 1e9, 1),
                        "frac_hbm": round(b / (t * 1e-3) / 1e9 / hbm, 4)}
        parts_out["sweep_per_n"] = per_n
        parts_out["sweep_min_frac_hbm"] = min(v["frac_hbm"] for v in per_n.values())
    for p in parts:
        gbs = bytes_[p] / (ms[p] * 1e-3) / 1e9
        parts_out[p] = {"ms": round(ms[p], 4), "gkeys_s": round(keys[p] / (ms[p] * 1e-3) / 1e9, 2),
                        "gb_s": round(gbs, 1), "frac_hbm": round(gbs / hbm, 4), "keys": keys[p], "bytes": bytes_[p]}
    total_keys = sum(keys[p] for p in parts)
    job_keys = sum_over_ranks([total_keys], dist, device)[0]  # ranks draw their own segment lengths

    result = {
        "metric": METRIC,
        "value": round(job_throughput(job_keys, ms["step"] * 1e-3) / 1e9, 3),
        "unit": "Gkeys/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms["step"], 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": config_dict(sizes, args.scale),
        "parts": parts_out,
        "roofline": {"bound": "hbm", "kernel": "fixed_tma_kernel (n=2..16, sweep)",
                     "achieved": round(sweep_gbs, 1), "peak": hbm, "peak_source": hbm_src,
                     "unit": "GB/s", "frac": round(sweep_gbs / hbm, 4),
                     "algorithmic_bytes": bytes_.get("sweep"),
                     "traffic": SWEEP_DRAM_BYTES if (args.scale == 0 and "sweep" in parts) else None,
                     "traffic_per": "one sweep step (15 launches, 2^24 arrays per n)",
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum at 2^22 arrays per n, "
                                       "reads scaled x4, writes x4 less the ~65 MB per launch still in L2"},
        "gpu_launches": launches_per_step(parts) * args.steps,
        "clocks": clocks,
        "wall_s_timed_loop": round(wall, 3),
    }

    result["config"]["launch_parameters"] = tuned or "library defaults"
    result["config"]["uneven_launch"] = ("replay of a captured CUDA graph (plan memset, plan / bin / tile / RSS "
                                         "kernels, scratch allocation nodes)" if graphs else "direct call")
    if not args.no_e2e:
        result["e2e"] = bench_e2e(args, sn, pristine, world, dist, device, parts)
    del work, graphs
    if "sweep" in parts and not args.no_families:
        result["network_families"] = bench_families(args, sn, pristine, device, dist)
    if not args.no_extras:
        result["extras"] = bench_extras(args, sn, device)
    if not args.no_configs:
        result["configs"] = bench_configs(args, sn, device)
    if not args.no_plain:
        result["plain_vs_batched"] = bench_plain_vs_batched(args, sn, device, dist)
    if rank == 0 and world == 1 and not args.no_serving:
        result["serving"] = bench_serving(args, device)
    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(sizes, budget_s=12.0)
    return result


def autotune(sn, keys, vals, offsets, rss_only=False):
    """sn_tune_segments (sn_tune_rss_segments if rss_only) on a batch; returns
    the installed parameters and the tuned time."""
    params, ms = sn.sn_tune_segments(keys, vals, offsets, rss_only=rss_only)
    return dict(params, tuned_ms=round(ms, 4))


def capture_uneven(sn, w):
    """The uneven-batch call captured once into a CUDA graph (same buffers every step)."""
    import torch
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        sn.check(sn.sn_sort_segments_u64(w["uneven_keys"], w["uneven_vals"], w["uneven_off"]), "capture")
    torch.cuda.current_stream().wait_stream(stream)
    return graph


# ------------------------------------------------------ network families ----

def _time_calls(fn, restore, reps, warm):
    """Mean CUDA-event time (ms) of fn() over `reps` runs, inputs restored before each."""
    import torch
    for _ in range(warm):
        restore()
        fn()
    times = []
    for _ in range(reps):
        restore()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.mean(times)


def bench_families(args, sn, pristine, device, dist):
    """Best known networks vs Bose-Nelson (Sec. 2.2.1, 4.3) on GB300: the u32
    sweep arrays (2^24 per n) and the paper's 16-byte items (u64 key + u64
    reference) at 2^22 arrays per n.  Both are HBM-bound here, so the table
    shows whether the extra comparators of Bose-Nelson cost anything."""
    import torch
    from paper_2002_05599_gb300 import workloads as wl
    hbm, _ = peaks()
    reps, warm = max(3, args.steps), max(3, args.warmup)
    out = {"u32_sweep": {}, "items16": {}, "timing": "CUDA events, mean over repetitions, inputs restored"}
    for n in SWEEP_NS:
        src = pristine[f"sweep{n}"]
        work = src.clone()
        row = {}
        for fam, name in ((sn.SN_NETWORK_BEST, "best"), (sn.SN_NETWORK_BOSE_NELSON, "bose_nelson")):
            ms = _time_calls(lambda: sn.check(sn.sn_sort_fixed_family(work, n, fam)), lambda: work.copy_(src),
                             reps, warm)
            row[name] = {"ms": round(ms, 4), "gkeys_s": round(src.numel() / (ms * 1e-3) / 1e9, 1),
                         "frac_hbm": round(8 * src.numel() / (ms * 1e-3) / 1e9 / hbm, 4)}
        out["u32_sweep"][n] = row
        del work
    count = (1 << 22) >> args.scale
    for n in (2, 4, 8, 12, 16):
        keys = wl.uniform_keys_torch(count * n, np.uint64, seed=500 + n, device=device)
        src = torch.stack([keys, torch.arange(count * n, dtype=torch.int64, device=device)], 1).reshape(-1)
        work = src.clone()
        row = {}
        for fam, name in ((sn.SN_NETWORK_BEST, "best"), (sn.SN_NETWORK_BOSE_NELSON, "bose_nelson")):
            ms = _time_calls(lambda: sn.check(sn.sn_sort_fixed_items(work, n, fam)), lambda: work.copy_(src),
                             reps, warm)
            row[name] = {"ms": round(ms, 4), "gitems_s": round(count * n / (ms * 1e-3) / 1e9, 1),
                         "frac_hbm": round(32 * count * n / (ms * 1e-3) / 1e9 / hbm, 4)}
        out["items16"][n] = row
        del keys, src, work
    sn.check(sn.sn_check(), "network families")
    out["items16_arrays_per_n"] = count
    return out


# --------------------------------------------- float keys, long segments ----

def bench_extras(args, sn, device):
    """Float keys next to the same-width unsigned keys (the order-preserving
    code runs in registers, so both should cost the same), and segments of
    257..4096 items (sn_sort_segments_large)."""
    import torch
    from paper_2002_05599_gb300 import workloads as wl
    hbm, _ = peaks()
    reps, warm = max(3, args.steps), max(3, args.warmup)
    out = {"timing": "CUDA events, mean over repetitions, inputs restored"}
    count = (1 << 24) >> args.scale
    fixed = {}
    for n in (8, 16):
        src = wl.uniform_keys_torch(count * n, np.uint32, seed=700 + n, device=device)
        work = src.clone()
        row = {}
        for name, fn in (("u32", sn.sn_sort_fixed), ("f32", sn.sn_sort_fixed_f32)):
            ms = _time_calls(lambda: sn.check(fn(work, n)), lambda: work.copy_(src), reps, warm)
            row[name] = {"ms": round(ms, 4), "gkeys_s": round(count * n / (ms * 1e-3) / 1e9, 1),
                         "frac_hbm": round(8 * count * n / (ms * 1e-3) / 1e9 / hbm, 4)}
        fixed[n] = row
        del src, work
    out["fixed_2^24_arrays"] = fixed
    nseg = (1 << 20) >> args.scale
    lens = wl.segment_lengths(nseg, "uniform", seed=701, lo=2, hi=256)
    off = wl.offsets_from_lengths(lens)
    d_off = torch.from_numpy(off.view(np.int32)).to(device)
    src = wl.uniform_keys_torch(int(off[-1]), np.uint32, seed=701, device=device)
    work = src.clone()
    row = {}
    for name, fn in (("u32", sn.sn_sort_segments), ("f32", sn.sn_sort_segments_f32)):
        ms = _time_calls(lambda: sn.check(fn(work, None, d_off)), lambda: work.copy_(src), reps, warm)
        row[name] = {"ms": round(ms, 4), "gkeys_s": round(src.numel() / (ms * 1e-3) / 1e9, 1)}
    out["segments_2^20_uniform_2..256_keys_only"] = row
    del src, work
    nseg = (1 << 16) >> args.scale
    lens = wl.segment_lengths(nseg, "uniform", seed=702, lo=257, hi=4096)
    off = wl.offsets_from_lengths(lens)
    d_off = torch.from_numpy(off.view(np.int32)).to(device)
    for dt, name, fn in ((np.uint32, "u32_keys_only", sn.sn_sort_segments_large),
                         (np.uint64, "u64_keys_only", sn.sn_sort_segments_large_u64)):
        src = wl.uniform_keys_torch(int(off[-1]), dt, seed=702, device=device)
        work = src.clone()
        ms = _time_calls(lambda: sn.check(fn(work, None, d_off)), lambda: work.copy_(src), reps, warm)
        out.setdefault(f"large_{nseg}_segments_257..4096", {})[name] = {
            "ms": round(ms, 4), "gkeys_s": round(src.numel() / (ms * 1e-3) / 1e9, 1)}
        del src, work
    # the rest of the RSS-range configuration: u64 keys, and Zipf(1.1) keys over 2^20 values
    nseg = (1 << 20) >> args.scale
    lens = wl.segment_lengths(nseg, "uniform", seed=101, lo=17, hi=256)
    off = wl.offsets_from_lengths(lens)
    d_off = torch.from_numpy(off.view(np.int32)).to(device)
    total = int(off[-1])
    variants = {}
    for name, dt, fn, dist in (("u32_uniform", np.uint32, sn.rss_sort_segments, "uniform"),
                               ("u32_zipf", np.uint32, sn.rss_sort_segments, "zipf"),
                               ("u64_uniform", np.uint64, sn.rss_sort_segments_u64, "uniform"),
                               ("u64_zipf", np.uint64, sn.rss_sort_segments_u64, "zipf")):
        if dist == "uniform":
            src = wl.uniform_keys_torch(total, dt, seed=101, device=device)
        else:
            src = wl.zipf_keys_torch(total, dtype=dt, seed=101, device=device)
        work = src.clone()
        ms = _time_calls(lambda: sn.check(fn(work, None, d_off)), lambda: work.copy_(src), reps, warm)
        kb = np.dtype(dt).itemsize
        variants[name] = {"ms": round(ms, 4), "gkeys_s": round(total / (ms * 1e-3) / 1e9, 2),
                          "frac_hbm": round((2 * kb * total + 4 * (nseg + 1)) / (ms * 1e-3) / 1e9 / hbm, 4)}
        del src, work
    out[f"rss_range_{nseg}_segments_17..256_keys_only"] = variants

    # one large array: sample-sort partition + segmented base case, next to torch.sort
    n = (1 << 26) >> args.scale
    src = wl.uniform_keys_torch(n, np.uint32, seed=703, device=device)
    work = src.clone()
    ms = _time_calls(lambda: sn.check(sn.sn_sort_large(work)), lambda: work.copy_(src), reps, warm)
    ref = src.to(torch.int64) & 0xFFFFFFFF  # torch sorts signed values: widen so the u32 order is kept
    ms_t = _time_calls(lambda: torch.sort(ref), lambda: None, reps, warm)
    out[f"large_sort_2^{26 - args.scale}_u32"] = {
        "sn_sort_large": {"ms": round(ms, 3), "gkeys_s": round(n / (ms * 1e-3) / 1e9, 2)},
        "torch.sort (int64 view, library reference point)": {"ms": round(ms_t, 3),
                                                             "gkeys_s": round(n / (ms_t * 1e-3) / 1e9, 2)}}
    del src, work, ref
    sn.check(sn.sn_check(), "extras")
    return out


# ------------------------------------------------ configurations ----------

def bench_configs(args, sn, device):
    """The configurations that are not parts of the step, each timed on its
    own: config 1 with a cold L2, config 2's other three key distributions,
    and the uneven batch with uniform 1..16 lengths (config 3 (i))."""
    import torch
    from paper_2002_05599_gb300 import workloads as wl
    hbm, _ = peaks()
    reps, warm = max(5, args.steps), max(3, args.warmup)
    out = {}

    # config 1: 2^20 arrays of 8 u32 keys, seed 1: 32 MiB, which fits in the
    # 126 MB L2, so a 256 MiB buffer is written after the input is restored
    # and before every timed launch
    count = (1 << 20) >> args.scale
    src = wl.uniform_keys_torch(count * 8, np.uint32, seed=1, device=device)
    work = src.clone()
    flush = torch.empty(64 << 20, dtype=torch.int32, device=device)
    times = []
    for rep in range(warm + reps):
        work.copy_(src)
        flush.fill_(rep)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        sn.check(sn.sn_sort_fixed(work, 8), "config 1")
        b.record()
        b.synchronize()
        if rep >= warm:
            times.append(a.elapsed_time(b))
    ms = statistics.median(times)
    out["config1_n8_2^20_arrays_cold_l2"] = {
        "ms": round(ms, 5), "gkeys_s": round(count * 8 / (ms * 1e-3) / 1e9, 1),
        "frac_hbm": round(8 * count * 8 / (ms * 1e-3) / 1e9 / hbm, 4), "reps": reps,
        "timing": "CUDA events around the one launch, median; 256 MiB written between restore and launch"}
    del src, work, flush

    # config 2: the sweep under each key distribution (uniform as in the step)
    count = (1 << 24) >> args.scale
    dists = {}
    for dist in ("uniform", "fewdistinct", "presorted", "reverse"):
        tot_ms, tot_b, worst = 0.0, 0, 1.0
        for n in SWEEP_NS:
            src = wl.uniform_keys_torch(count * n, np.uint32, seed=900 + n, device=device)
            if dist == "fewdistinct":
                src = src & 3
            elif dist in ("presorted", "reverse"):
                w = torch.sort(src.view(-1, n).to(torch.int64) & 0xFFFFFFFF, dim=1).values
                if dist == "reverse":
                    w = w.flip(1)
                src = torch.where(w >= (1 << 31), w - (1 << 32), w).to(torch.int32).reshape(-1)
            work = src.clone()
            ms = _time_calls(lambda: sn.check(sn.sn_sort_fixed(work, n)), lambda: work.copy_(src), reps, warm)
            tot_ms += ms
            tot_b += 8 * count * n
            worst = min(worst, 8 * count * n / (ms * 1e-3) / 1e9 / hbm)
            del src, work
        dists[dist] = {"ms": round(tot_ms, 4), "frac_hbm": round(tot_b / (tot_ms * 1e-3) / 1e9 / hbm, 4),
                       "min_frac_hbm_over_n": round(worst, 4)}
    out["config2_sweep_by_distribution"] = dists

    # config 3 (i): 2^24 segments, lengths uniform 1..16, u64 keys + u32 payload
    nseg = (1 << 24) >> args.scale
    lens = wl.segment_lengths(nseg, "uniform", seed=1, lo=1, hi=16)
    off = wl.offsets_from_lengths(lens)
    total = int(off[-1])
    d_off = torch.from_numpy(off.view(np.int32)).to(device)
    keys = wl.uniform_keys_torch(total, np.uint64, seed=1, device=device)
    vals = torch.arange(total, dtype=torch.int32, device=device)
    wk, wv = keys.clone(), vals.clone()
    tuned = "library defaults"
    if not args.no_tune:
        tuned = autotune(sn, wk, wv, d_off)

    def restore():
        wk.copy_(keys)
        wv.copy_(vals)

    ms = _time_calls(lambda: sn.check(sn.sn_sort_segments_u64(wk, wv, d_off)), restore, reps, warm)
    byt = 24 * total + 4 * (nseg + 1)
    out["config3i_uniform_1..16_u64_keys_u32_payload"] = {
        "segments": nseg, "items": total, "ms": round(ms, 4), "gkeys_s": round(total / (ms * 1e-3) / 1e9, 2),
        "gb_s": round(byt / (ms * 1e-3) / 1e9, 1), "frac_hbm": round(byt / (ms * 1e-3) / 1e9 / hbm, 4),
        "launch_parameters": tuned}
    del keys, vals, wk, wv
    sn.check(sn.sn_check(), "configs")
    return out


# ------------------------------------------------- plain vs batched ---------

def bench_plain_vs_batched(args, sn, device, dist):
    """The same arrays sorted two ways: plain = grouped by length into
    contiguous fixed-n arrays, one sn_sort_fixed launch per n; batched = the
    CSR batch in its original interleaved order, one sn_sort_segments call.
    Lengths uniform 1..16 (length-1 segments need no work in either form)."""
    import torch
    from paper_2002_05599_gb300 import workloads as wl
    nseg = (1 << 24) >> args.scale
    out = {"workload": f"{nseg} segments, lengths uniform 1..16, keys only, uniform keys (seed 3)",
           "timing": "CUDA events per call sequence, mean of the timed repetitions; "
                     "inputs restored from pristine copies between repetitions"}
    lens = wl.segment_lengths(nseg, "uniform", seed=3, lo=1, hi=16)
    off = wl.offsets_from_lengths(lens)
    total = int(off[-1])
    d_off = torch.from_numpy(off.view(np.int32)).to(device)
    # plain layout: segments grouped by length, each length's block of arrays
    # starting on a 16-byte boundary like a buffer of its own (built once, untimed)
    counts = np.bincount(lens, minlength=17)
    order = np.argsort(lens, kind="stable")
    starts = off[:-1][order].astype(np.int64)
    glens = lens[order].astype(np.int64)
    gather = np.repeat(starts, glens) + (np.arange(total) - np.repeat(np.cumsum(glens) - glens, glens))
    block_at, at = {}, 0
    for n in range(1, 17):
        at = (at + 3) & ~3  # 16 bytes for u32 keys, 32 for u64: aligned either way
        block_at[n] = at
        at += int(counts[n]) * n
    place = np.concatenate([np.arange(block_at[n], block_at[n] + int(counts[n]) * n) for n in range(1, 17)])
    d_gather = torch.from_numpy(gather).to(device)
    d_place = torch.from_numpy(place).to(device)
    padded = at
    for dtype, name, fixed, seg in ((np.uint64, "u64", sn.sn_sort_fixed_u64, sn.sn_sort_segments_u64),
                                    (np.uint32, "u32", sn.sn_sort_fixed, sn.sn_sort_segments)):
        keys = wl.uniform_keys_torch(total, dtype, seed=3, device=device)
        grouped = torch.zeros(padded, dtype=keys.dtype, device=device)
        grouped[d_place] = keys[d_gather]
        work_b, work_p = keys.clone(), grouped.clone()
        views = {n: work_p[block_at[n]:block_at[n] + int(counts[n]) * n] for n in range(1, 17)}

        def plain():
            for n in range(2, 17):
                if counts[n]:
                    sn.check(fixed(views[n], n, int(counts[n])), f"plain n={n}")

        def batched():
            sn.check(seg(work_b, None, d_off), "batched")

        tuning = "library defaults"
        if not args.no_tune:
            work_b.copy_(keys)
            tuning = autotune(sn, work_b, None, d_off)

        def plain_from_csr():  # what a caller holding the CSR batch has to do for the plain form
            work_p[d_place] = work_b[d_gather]
            plain()
            work_b[d_gather] = work_p[d_place]

        res = {}
        for label, fn, src, dst in (("plain", plain, grouped, work_p), ("batched", batched, keys, work_b),
                                    ("plain_from_csr", plain_from_csr, keys, work_b)):
            for _ in range(max(3, args.warmup)):
                dst.copy_(src)
                fn()
            times = []
            for _ in range(max(3, args.steps)):
                dst.copy_(src)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                b.record()
                b.synchronize()
                times.append(a.elapsed_time(b))
            res[label] = statistics.mean(times)
        sn.check(sn.sn_check(), "plain vs batched")
        # both forms sort the same arrays: compare through the grouping
        work_b.copy_(keys)
        batched()
        work_p.copy_(grouped)
        plain()
        assert torch.equal(work_b[d_gather], work_p[d_place]), "plain and batched results differ"
        ms_p, ms_b, ms_c = max_over_ranks([res["plain"], res["batched"], res["plain_from_csr"]], dist, device)
        out[name] = {"plain_ms": round(ms_p, 4), "plain_gkeys_s": round(total / (ms_p * 1e-3) / 1e9, 2),
                     "plain_launches": int(sum(1 for n in range(2, 17) if counts[n])),
                     "batched_ms": round(ms_b, 4), "batched_gkeys_s": round(total / (ms_b * 1e-3) / 1e9, 2),
                     "batched_launches": 4, "batched_over_plain": round(ms_p / ms_b, 3),
                     "plain_from_csr_ms": round(ms_c, 4),
                     "plain_from_csr_gkeys_s": round(total / (ms_c * 1e-3) / 1e9, 2),
                     "plain_from_csr_note": "group the CSR batch by length (gather), one launch per n, "
                                            "scatter back (torch indexing for the data movement)",
                     "batched_over_plain_from_csr": round(ms_c / ms_b, 3),
                     "batched_launch_parameters": tuning}
        del keys, grouped, work_b, work_p, views
    return out


# ----------------------------------------------------------- serving --------

def bench_serving(args, device):
    """Continuous batching under a Poisson request stream: requests of
    log-uniform 1..10^5 segments (lengths uniform 2..256, u32 uniform keys) in
    pinned host memory, served by the library's request server under a 40 GB
    device budget; latency = arrival -> sorted keys back in host memory."""
    import ctypes
    import torch
    from paper_2002_05599_gb300 import workloads as wl
    from paper_2002_05599_gb300.server import SortServer, _lib, now_ns
    pool_nseg = (1 << 22) >> args.scale
    lens = wl.segment_lengths(pool_nseg, "uniform", seed=7, lo=2, hi=256)
    off = wl.offsets_from_lengths(lens)
    total = int(off[-1])
    keys_in = torch.empty(total, dtype=torch.int32, pin_memory=True)
    keys_in.copy_(wl.uniform_keys_torch(total, np.uint32, seed=7, device=device))
    keys_out = torch.empty(total, dtype=torch.int32, pin_memory=True)
    off_h = torch.from_numpy(off.view(np.int32)).pin_memory()
    rng = np.random.default_rng(1)
    n_req = max(1, int(args.serve_rate * args.serve_seconds))
    arrivals = np.cumsum(rng.exponential(1.0 / args.serve_rate, n_req))
    max_cnt = min(100_000, pool_nseg)
    counts = np.floor(np.exp(rng.uniform(0.0, np.log(max_cnt + 1), n_req))).astype(np.int64).clip(1, max_cnt)
    starts = rng.integers(0, pool_nseg - counts + 1)
    tuning = "library defaults"
    if not args.no_tune:  # tune on the first 10^6 pool segments (same length mix)
        import paper_2002_05599_gb300 as sn
        m = min(pool_nseg, 1_000_000)
        dk = keys_in[:int(off[m])].to(device)
        tuning = autotune(sn, dk, None, torch.from_numpy(off[:m + 1].view(np.int32)).to(device))
        del dk
    budget = 40 << 30
    srv = SortServer(budget_bytes=budget, key_bytes=4, slots=4)
    lib, h = _lib(), srv._h
    kin, kout, offp = keys_in.data_ptr(), keys_out.data_ptr(), off_h.data_ptr()
    ticket = ctypes.c_uint64()

    def stream(n, t0):
        lag = 0
        for i in range(n):
            due = t0 + int(arrivals[i] * 1e9)
            while now_ns() < due:
                pass
            lag = max(lag, now_ns() - due)
            rc = lib.sn_server_submit(h, kin, None, offp + 4 * int(starts[i]), int(counts[i]), kout, None, due,
                                      ctypes.byref(ticket))
            if rc != 0:
                raise RuntimeError(f"submit failed: {rc}")
        srv.drain()
        return lag

    stream(min(n_req, 200), now_ns() + 1_000_000)  # warm-up: device set-up, first batches
    srv.stats(reset=True)
    lag = stream(n_req, now_ns() + 2_000_000)
    st = srv.stats()
    srv.close()
    keys_req = float(np.sum(off[starts + counts].astype(np.int64) - off[starts].astype(np.int64)))
    span = float(arrivals[-1])
    return {"requests": n_req, "rate_hz": args.serve_rate, "seconds": round(span, 3),
            "segments_per_request": "log-uniform 1..1e5", "segment_lengths": "uniform 2..256",
            "keys": "u32 uniform, pinned host memory", "budget_gb": budget / 2**30, "slots": 4,
            "launch_parameters": tuning,
            "offered_gkeys_s": round(keys_req / span / 1e9, 2),
            "achieved_gkeys_s": round(st["keys_per_s"] / 1e9, 2),
            "p50_ms": round(st["latency_p50_us"] / 1e3, 3), "p99_ms": round(st["latency_p99_us"] / 1e3, 3),
            "max_ms": round(st["latency_max_us"] / 1e3, 3), "mean_ms": round(st["latency_mean_us"] / 1e3, 3),
            "completed": st["completed"], "failed": st["failed"], "batches": st["batches"],
            "max_requests_per_batch": st["max_batch_requests_seen"], "max_batches_in_flight": st["max_inflight_seen"],
            "peak_device_gb": round(st["peak_device_bytes"] / 2**30, 3), "client_max_lag_ms": round(lag / 1e6, 3)}


def e2e_jobs(sn, host, out, dev, parts):
    """The step cut into jobs of (host->device copies, sorts, device->host
    copies): one per fixed n, the uneven batch in 4 and the RSS range in 2
    contiguous segment ranges (offsets stay absolute: a range is sorted by
    passing the offsets from its first segment)."""
    jobs = []
    if "sweep" in parts:
        for n in SWEEP_NS:
            k = f"sweep{n}"
            jobs.append(([(host[k], dev[k])], lambda s, k=k, n=n: sn.check(sn.sn_sort_fixed(dev[k], n, stream=s)),
                         [(dev[k], out[k])]))
    for part, nchunks, fn in (("uneven", 4, sn.sn_sort_segments_u64), ("rss", 2, sn.rss_sort_segments)):
        if part not in parts:
            continue
        off_h = host[f"{part}_off"].numpy().view(np.uint32)
        nseg = off_h.size - 1
        keys, vals = f"{part}_keys", f"{part}_vals"
        for c in range(nchunks):
            a, b = nseg * c // nchunks, nseg * (c + 1) // nchunks
            ea, eb = int(off_h[a]), int(off_h[b])
            h2d = [(host[f"{part}_off"][a:b + 1], dev[f"{part}_off"][a:b + 1]),
                   (host[keys][ea:eb], dev[keys][ea:eb])]
            d2h = [(dev[keys][ea:eb], out[keys][ea:eb])]
            if vals in host:
                h2d.append((host[vals][ea:eb], dev[vals][ea:eb]))
                d2h.append((dev[vals][ea:eb], out[vals][ea:eb]))

            def run(s, a=a, b=b, keys=keys, vals=vals, fn=fn, part=part):
                sn.check(fn(dev[keys], dev.get(vals), dev[f"{part}_off"][a:b + 1], b - a, stream=s), part)
            jobs.append((h2d, run, d2h))
    return jobs


def e2e_check(host, out, parts, samples=2000):
    """Spot check of the pipelined results on the host: sampled arrays and
    segments must equal numpy's sort of the same input."""
    rng = np.random.default_rng(5)
    u = {4: np.uint32, 8: np.uint64}
    if "sweep" in parts:
        for n in SWEEP_NS:
            k = f"sweep{n}"
            src = host[k].numpy().view(u[host[k].element_size()]).reshape(-1, n)
            got = out[k].numpy().view(u[out[k].element_size()]).reshape(-1, n)
            rows = rng.integers(0, src.shape[0], samples)
            if not np.array_equal(np.sort(src[rows], axis=1), got[rows]):
                raise RuntimeError(f"e2e result differs for n={n}")
    for part in ("uneven", "rss"):
        if part not in parts:
            continue
        off = host[f"{part}_off"].numpy().view(np.uint32)
        kk = f"{part}_keys"
        src = host[kk].numpy().view(u[host[kk].element_size()])
        got = out[kk].numpy().view(u[out[kk].element_size()])
        for i in rng.integers(0, off.size - 1, samples):
            a, b = int(off[i]), int(off[i + 1])
            if not np.array_equal(np.sort(src[a:b]), got[a:b]):
                raise RuntimeError(f"e2e result differs in {part} segment {i}")


def bench_e2e(args, sn, pristine, world, dist, device, parts=PARTS):
    """The same step through the C ABI with host buffers (pinned): per job,
    host->device copies on one stream, the sorts on a second, device->host
    copies on a third, so the copies of one job overlap the sorts of another.
    Steps alternate between two device buffer sets, so that a step's
    host->device copies overlap the previous step's sorts and device->host
    copies (a set is refilled once the step before last has read it out)."""
    import torch
    host = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in pristine.items()}
    for k, v in pristine.items():
        host[k].copy_(v)
    out = {k: torch.empty_like(host[k], pin_memory=True) for k in host if not k.endswith("_off")}
    devs = [{k: torch.empty_like(v) for k, v in pristine.items()} for _ in range(2)]
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = sum(t.numel() * t.element_size() for t in out.values())
    keys = sum(part_keys(pristine).values())
    jobsets = [e2e_jobs(sn, host, out, dev, parts) for dev in devs]
    s_h, s_c, s_d = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    read_out = [torch.cuda.Event(), torch.cuda.Event()]  # set b's results copied out
    for ev in read_out:
        ev.record(s_d)

    def step(i):
        b = i % 2
        s_h.wait_event(read_out[b])
        for hd, run, dh in jobsets[b]:
            with torch.cuda.stream(s_h):
                for src, dst in hd:
                    dst.copy_(src, non_blocking=True)
            s_c.wait_stream(s_h)
            run(s_c)
            s_d.wait_stream(s_c)
            with torch.cuda.stream(s_d):
                for src, dst in dh:
                    dst.copy_(src, non_blocking=True)
        read_out[b].record(s_d)

    step(0)
    torch.cuda.synchronize()
    e2e_check(host, out, parts)
    steps = max(2, min(args.steps, 6))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        step(1 + i)
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / steps
    e2e_check(host, out, parts, samples=200)
    sec = max_over_ranks([sec], dist, device)[0]
    job_keys = sum_over_ranks([keys], dist, device)[0]
    sn.check(sn.sn_check(), "e2e")
    return {"value": round(job_throughput(job_keys, sec) / 1e9, 3), "unit": "Gkeys/s", "ms_per_step": round(sec * 1e3, 3),
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "pipeline": f"{len(jobsets[0])} jobs a step; H2D, sorts and D2H on three streams; "
                        "two device buffer sets, alternate steps"}


# ----------------------------------------------------------- CPU oracle -----

def oracle_sample(sizes, frac_shift):
    """A bounded sample of the step: the same workloads, 2^-frac_shift of the units."""
    from paper_2002_05599_gb300 import workloads as wl
    sample = {}
    cnt = max(1, sizes["sweep_count"] >> frac_shift)
    for n in SWEEP_NS:
        sample[f"sweep{n}"] = wl.fixed_arrays(n, cnt, "uniform", np.uint32, seed=1000 + n)
    k, v, off = wl.segment_batch(max(1, sizes["uneven_nseg"] >> frac_shift), "geometric", "uniform", np.uint64,
                                 True, seed=1, p=0.15, cap=256)
    sample["uneven"] = (k, v, off)
    k, _, off = wl.segment_batch(max(1, sizes["rss_nseg"] >> frac_shift), "uniform", "uniform", np.uint32,
                                 False, seed=101, lo=17, hi=256)
    sample["rss"] = (k, None, off)
    desc = (f"2^-{frac_shift} of every part: {cnt} arrays per n, "
            f"{sample['uneven'][2].size - 1} uneven segments, {sample['rss'][2].size - 1} RSS segments")
    return sample, desc


def oracle_step(sample):
    import oracle
    keys = 0
    t0 = time.perf_counter()
    for n in SWEEP_NS:
        a = sample[f"sweep{n}"]
        oracle.sort_fixed(a, n)
        keys += a.size
    for part in ("uneven", "rss"):
        k, v, off = sample[part]
        oracle.sort_segments(k, v, off)
        keys += k.size
    return keys, time.perf_counter() - t0


def _split_sample(sample, parts):
    """The sample cut into `parts` independent pieces (array ranges; segment
    ranges with their offsets rebased), so that several threads can run the
    oracle on it (ctypes releases the GIL during each oracle call)."""
    pieces = [dict() for _ in range(parts)]
    for n in SWEEP_NS:
        a = sample[f"sweep{n}"].reshape(-1, n)
        for i, chunk in enumerate(np.array_split(a, parts)):
            pieces[i][f"sweep{n}"] = chunk.reshape(-1)
    for part in ("uneven", "rss"):
        k, v, off = sample[part]
        bounds = np.linspace(0, off.size - 1, parts + 1).astype(np.int64)
        for i in range(parts):
            s0, s1 = int(bounds[i]), int(bounds[i + 1])
            a, b = int(off[s0]), int(off[s1])
            pieces[i][part] = (k[a:b], None if v is None else v[a:b], (off[s0:s1 + 1] - off[s0]).astype(np.uint32))
    return pieces


def oracle_step_threads(pieces):
    """oracle_step over the pieces on one thread each; (keys, seconds)."""
    from concurrent.futures import ThreadPoolExecutor
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=len(pieces)) as ex:
        keys = sum(k for k, _ in ex.map(oracle_step, pieces))
    return keys, time.perf_counter() - t0


def _sized_sample(sizes, budget_s, threads, shift=9):
    """The largest 2^-shift sample that a probe predicts to take at most
    budget_s seconds on `threads` threads."""
    import math
    sample, desc = oracle_sample(sizes, shift)
    _, probe = oracle_step(sample)
    grow = int(math.floor(math.log2(max(1.0, budget_s * threads / max(probe, 1e-6)))))
    shift = max(0, shift - grow)
    return oracle_sample(sizes, shift)


def cpu_baseline(sizes, budget_s=15.0):
    """The oracle on the host: on one core (the paper's single-core
    measurement), and on every core of the host (one thread per core over
    independent pieces of the sample), each on the largest 2^-shift sample of
    the step that a probe predicts to take at most `budget_s` seconds."""
    import oracle
    oracle.build()
    sample, desc = _sized_sample(sizes, budget_s, 1)
    keys, sec = oracle_step(sample)
    one = {"value": round(keys / sec / 1e9, 5), "cores": 1, "sample": desc, "seconds": round(sec, 3)}
    del sample
    cores = os.cpu_count() or 1
    sample, desc_all = _sized_sample(sizes, budget_s, cores)
    keys, sec = oracle_step_threads(_split_sample(sample, cores))
    return {"value": round(keys / sec / 1e9, 5), "unit": "Gkeys/s", "cores": cores, "kind": "oracle",
            "sample": desc_all + f"; {cores} threads (os.cpu_count()), one per piece of the sample",
            "seconds": round(sec, 3), "single_core": one}


def bench_reference(args, rank, world):
    """--impl reference: the CPU oracle, timed on the host, on a bounded sample."""
    import oracle
    oracle.build()
    sizes = workload_sizes(args.scale)
    cores = os.cpu_count() or 1
    sample, desc = oracle_sample(sizes, 10)
    _, probe = oracle_step(sample)
    # keep the whole run (warm-up + timed, one thread per core) within about two minutes
    shift = 10
    while shift > 4 and probe * 2 * (args.steps + args.warmup) < 120 * cores:
        shift -= 1
        sample, desc = oracle_sample(sizes, shift)
        _, probe = oracle_step(sample)
    pieces = _split_sample(sample, cores)
    desc += f"; {cores} threads (os.cpu_count()), one per piece of the sample"
    for _ in range(args.warmup):
        oracle_step_threads(pieces)
    times, keys = [], 0
    for _ in range(args.steps):
        keys, sec = oracle_step_threads(pieces)
        times.append(sec)
    sec = statistics.mean(times)
    value = round(keys / sec / 1e9, 5)
    return {
        "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": config_dict(sizes, args.scale), "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "Gkeys/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(bench_reference(args, rank, world)), flush=True)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
        dist = tdist
    res = bench_ours(args, rank, world, local_rank, dist)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
