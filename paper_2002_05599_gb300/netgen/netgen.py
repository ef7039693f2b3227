"""Sorting-network table generator (build-time tool).

Emits the comparator lists the CUDA kernels unroll:

* ``csrc/networks_gen.h`` -- one X-macro per n = 2..16 listing the comparators
  ``CE(i, j)`` (0-based channels, i < j, the smaller value goes to i,
  Sec. 2.1) in execution order, plus the XOR-mask schedule of the 32-lane
  warp network;
* ``netgen/networks.json`` -- the same lists with size, depth and provenance.

Where the networks come from:

* n = 16 and n = 10: the networks the paper prints (Figure network:best:16, 60
  comparators in ten levels; Figure network:optimal:10, 29 comparators in nine
  levels, Sec. 2.1-2.2), kept as seed data below;
* smaller n: channels are removed from those two networks by feeding +inf into
  the top channel (or -inf into the bottom one), deleting every comparator the
  sentinel meets and untangling the reversed comparators this leaves (Knuth,
  TAOCP vol. 3, Sec. 5.3.4, exercise 16);
* n = 8: Batcher's odd-even merge sort (19 comparators);
* n = 11..13: the best of pruning, the randomised greedy search in
  ``search.c`` and the evolutionary search in ``evolve.c`` (results stored in
  ``searched.json`` with the arguments that reproduce them; n = 13 from
  ``evolve.c``, 45 comparators);
* the warp network for 17..32 items: Batcher's bitonic sorter written with
  ascending comparators only (the first step of each merge compares mirrored
  positions, partner ``i ^ (k - 1)``; later steps use ``i ^ j``).

Every emitted network is checked here on all 2^n 0-1 inputs (0-1 principle)
before anything is written.

usage: python -m paper_2002_05599_gb300.netgen.netgen [--check] [--search N ...]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.dirname(HERE)
HEADER = os.path.join(PKG, "csrc", "networks_gen.h")
JSON_OUT = os.path.join(HERE, "networks.json")
SEARCHED = os.path.join(HERE, "searched.json")

# Best-known sizes for n = 2..16 from the sorting-network literature; the
# paper confirms n = 10 (29, optimal) and n = 16 (60, printed network).
BEST_KNOWN_SIZE = {2: 1, 3: 3, 4: 5, 5: 9, 6: 12, 7: 16, 8: 19, 9: 25, 10: 29,
                   11: 35, 12: 39, 13: 45, 14: 51, 15: 56, 16: 60}

# The paper's printed networks, 1-based channels as drawn, level by level.
_PAPER_BEST16 = [
    [(1, 2), (3, 4), (5, 6), (7, 8), (9, 10), (11, 12), (13, 14), (15, 16)],
    [(1, 3), (5, 7), (9, 11), (13, 15), (2, 4), (6, 8), (10, 12), (14, 16)],
    [(1, 5), (9, 13), (2, 6), (10, 14), (3, 7), (11, 15), (4, 8), (12, 16)],
    [(1, 9), (2, 10), (3, 11), (4, 12), (5, 13), (6, 14), (7, 15), (8, 16)],
    [(6, 11), (7, 10), (4, 13), (14, 15), (8, 12), (2, 3), (5, 9)],
    [(2, 5), (8, 14), (3, 9), (12, 15)],
    [(3, 5), (6, 7), (10, 11), (12, 14), (4, 9), (8, 13)],
    [(7, 9), (11, 13), (4, 6), (8, 10)],
    [(4, 5), (6, 7), (8, 9), (10, 11), (12, 13)],
    [(7, 8), (9, 10)],
]
_PAPER_OPT10 = [
    [(5, 10), (4, 9), (3, 8), (2, 7), (1, 6)],
    [(2, 5), (7, 10), (1, 4), (6, 9)],
    [(1, 3), (4, 7), (8, 10)],
    [(1, 2), (3, 5), (6, 8), (9, 10)],
    [(2, 3), (5, 7), (8, 9), (4, 6)],
    [(3, 6), (7, 9), (2, 4), (5, 8)],
    [(3, 4), (7, 8)],
    [(4, 5), (6, 7)],
    [(5, 6)],
]


def _flatten0(levels):
    return [(i - 1, j - 1) for lv in levels for (i, j) in lv]


PAPER_BEST16 = _flatten0(_PAPER_BEST16)
PAPER_OPT10 = _flatten0(_PAPER_OPT10)


# ----------------------------------------------------------------- checks ----

def sorts_all_01(n: int, net) -> bool:
    """True iff the network sorts all 2^n 0-1 inputs (bit i = channel i)."""
    full = (1 << n) - 1
    sorted_vectors = {full ^ ((1 << (n - t)) - 1) for t in range(n + 1)}
    for v in range(1 << n):
        for i, j in net:
            if (v >> i) & 1 and not (v >> j) & 1:
                v ^= (1 << i) | (1 << j)
        if v not in sorted_vectors:
            return False
    return True


def depth(n: int, net) -> int:
    last = [0] * n
    d = 0
    for i, j in net:
        lv = max(last[i], last[j]) + 1
        last[i] = last[j] = lv
        d = max(d, lv)
    return d


# ------------------------------------------------------------ construction ----

def untangle(net):
    """Turn a network whose comparators may be reversed (min -> first channel
    even when it is the larger index) into a standard one: flip the first
    reversed comparator and exchange its two channel labels in every later
    comparator; repeat (Knuth 5.3.4, ex. 16)."""
    net = [list(c) for c in net]
    for k in range(len(net)):
        a, b = net[k]
        if a > b:
            net[k] = [b, a]
            for later in net[k + 1:]:
                for t in range(2):
                    if later[t] == a:
                        later[t] = b
                    elif later[t] == b:
                        later[t] = a
    return [tuple(c) for c in net]


def remove_channel(n: int, net, top: bool):
    """Network on n-1 channels: feed +inf into channel n-1 (top) or -inf into
    channel 0 (bottom) and drop the comparators the sentinel passes through.

    Data never moves for the sentinel; instead the two channel names are
    exchanged when a comparator would have moved it.  ``where[name]`` is the
    wire that currently carries channel ``name``."""
    wire_s = n - 1 if top else 0
    where = list(range(n))
    kept = []
    for i, j in net:
        a, b = where[i], where[j]
        if top:
            if a == wire_s:            # +inf on the min side: it would move to j
                where[i], where[j] = b, a
                continue
            if b == wire_s:            # +inf already on the max side
                continue
        else:
            if b == wire_s:            # -inf on the max side: it would move to i
                where[i], where[j] = b, a
                continue
            if a == wire_s:
                continue
        kept.append((a, b))
    # output channel k (excluding the sentinel's) is read from wire where[k]
    names = [k for k in range(n) if where[k] != wire_s]
    wire_to_new = {}
    for new, k in enumerate(names):
        wire_to_new[where[k]] = new
    relabelled = [(wire_to_new[a], wire_to_new[b]) for a, b in kept]
    return untangle(relabelled)


def batcher_odd_even(n: int):
    """Batcher's odd-even merge sort on n = 2^p channels."""
    pairs = []

    def merge(lo: int, hi: int, r: int) -> None:
        step = 2 * r
        if step < hi - lo:
            merge(lo, hi, step)
            merge(lo + r, hi, step)
            for i in range(lo + r, hi - r, step):
                pairs.append((i, i + r))
        else:
            pairs.append((lo, lo + r))

    def sort(lo: int, hi: int) -> None:
        if hi - lo >= 1:
            mid = lo + (hi - lo) // 2
            sort(lo, mid)
            sort(mid + 1, hi)
            merge(lo, hi, 1)

    sort(0, n - 1)
    return pairs


def bose_nelson(n: int):
    """Bose and Nelson's recursive construction (1962), 0-based comparators in
    the recursion's emission order (the order the paper calls locality-
    optimised, BN-L): sort the first half and the second half, then merge
    them with the recursive two-sequence merge."""
    pairs = []

    def merge(i: int, x: int, j: int, y: int) -> None:
        # merge the sorted runs [i, i + x) and [j, j + y)
        if x == 1 and y == 1:
            pairs.append((i, j))
        elif x == 1 and y == 2:
            pairs.append((i, j + 1))
            pairs.append((i, j))
        elif x == 2 and y == 1:
            pairs.append((i, j))
            pairs.append((i + 1, j))
        else:
            a = x // 2
            b = y // 2 if x % 2 else (y + 1) // 2
            merge(i, a, j, b)
            merge(i + a, x - a, j + b, y - b)
            merge(i + a, x - a, j, b)

    def sort(i: int, m: int) -> None:
        if m > 1:
            a = m // 2
            sort(i, a)
            sort(i + a, m - a)
            merge(i, a, i + a, m - a)

    sort(0, n)
    return pairs


def by_levels(net):
    """The same comparators emitted level by level (as-soon-as-possible depth,
    the order the paper calls parallelism-optimised, BN-P); stable within a
    level."""
    avail = {}
    level_of = []
    for a, b in net:
        lv = max(avail.get(a, 0), avail.get(b, 0))
        level_of.append(lv)
        avail[a] = avail[b] = lv + 1
    order = sorted(range(len(net)), key=lambda k: (level_of[k], k))
    return [net[k] for k in order]


def warp_schedule(width: int = 32):
    """XOR masks of the ascending bitonic sorter on ``width`` lanes."""
    masks = []
    k = 2
    while k <= width:
        masks.append(k - 1)          # mirrored compare within blocks of k
        j = k // 4
        while j >= 1:
            masks.append(j)
            j //= 2
        k *= 2
    return masks


def schedule_pairs(masks, width: int = 32):
    return [(i, i ^ m) for m in masks for i in range(width) if i < (i ^ m)]


def _searched():
    if not os.path.exists(SEARCHED):
        return []
    with open(SEARCHED) as f:
        return json.load(f)


def pruned_candidates():
    """All networks reachable by removing top/bottom channels from the paper's
    n = 16 and n = 10 networks: {n: [(net, provenance)]}."""
    out = {}
    seen = set()
    frontier = [(16, PAPER_BEST16, "paper16"), (10, PAPER_OPT10, "paper10"),
                (8, batcher_odd_even(8), "batcher-odd-even")]
    for rec in _searched():
        frontier.append((rec["n"], [tuple(p) for p in rec["pairs"]], rec["provenance"]))
    while frontier:
        nxt = []
        for n, net, prov in frontier:
            key = (n, tuple(net))
            if key in seen:
                continue
            seen.add(key)
            out.setdefault(n, []).append((net, prov))
            if n > 2:
                nxt.append((n - 1, remove_channel(n, net, True), prov + "-top"))
                nxt.append((n - 1, remove_channel(n, net, False), prov + "-bottom"))
        frontier = nxt
    return out


def choose_networks():
    """Best network per n = 2..16 (fewest comparators, then smallest depth)."""
    cands = pruned_candidates()
    for rec in _searched():
        cands.setdefault(rec["n"], []).append(
            ([tuple(p) for p in rec["pairs"]], rec["provenance"]))
    chosen = {}
    for n in range(2, 17):
        best = None
        for net, prov in cands.get(n, []):
            key = (len(net), depth(n, net))
            if best is None or key < best[0]:
                best = (key, net, prov)
        if best is None:
            raise RuntimeError(f"no network for n={n}")
        chosen[n] = {"pairs": best[1], "provenance": best[2]}
    return chosen


# ------------------------------------------------------------------ output ----

def render(chosen, masks) -> tuple[str, str]:
    lines = [
        "/* Generated by paper_2002_05599_gb300/netgen/netgen.py -- do not edit.",
        " *",
        " * SN_NET_<n>(CE) expands to CE(i, j) for every comparator of the n-channel",
        " * sorting network in execution order: channels are 0-based, i < j, and the",
        " * comparator leaves the smaller value on channel i (Sec. 2.1).  Every",
        " * network was checked on all 2^n 0-1 inputs by the generator.",
        " */",
        "#pragma once",
        "",
    ]
    for n in range(2, 17):
        net = chosen[n]["pairs"]
        body = " ".join(f"CE({i},{j})" for i, j in net)
        lines.append(f"/* n={n}: {len(net)} comparators, depth {depth(n, net)}, "
                     f"from {chosen[n]['provenance']} */")
        lines.append(f"#define SN_NET_SIZE_{n} {len(net)}")
        lines.append(f"#define SN_NET_{n}(CE) {body}")
        lines.append("")
    lines.append("/* Bose-Nelson networks (recursive construction, emission order of the")
    lines.append(" * recursion): SN_BN_<n>(CE), same conventions as SN_NET_<n>. */")
    for n in range(2, 17):
        net = bose_nelson(n)
        body = " ".join(f"CE({i},{j})" for i, j in net)
        lines.append(f"/* n={n}: {len(net)} comparators, depth {depth(n, net)} */")
        lines.append(f"#define SN_BN_SIZE_{n} {len(net)}")
        lines.append(f"#define SN_BN_{n}(CE) {body}")
    lines.append("")
    lines.append("/* 32-lane warp network (17..32 items): lane l exchanges with lane l ^ M at")
    lines.append(" * each step M below; the lower lane keeps the smaller item. */")
    lines.append(f"#define SN_WARP32_STEPS {len(masks)}")
    lines.append("#define SN_WARP32_SCHEDULE(STEP) " + " ".join(f"STEP({m})" for m in masks))
    lines.append("")
    header = "\n".join(lines)
    data = {
        "networks": {str(n): {"pairs": [list(p) for p in chosen[n]["pairs"]],
                              "size": len(chosen[n]["pairs"]),
                              "depth": depth(n, chosen[n]["pairs"]),
                              "best_known_size": BEST_KNOWN_SIZE[n],
                              "provenance": chosen[n]["provenance"]}
                     for n in range(2, 17)},
        "warp32": {"masks": masks, "pairs": [list(p) for p in schedule_pairs(masks)]},
        "bose_nelson": {str(n): {"pairs": [list(p) for p in bose_nelson(n)], "size": len(bose_nelson(n)),
                                 "depth": depth(n, bose_nelson(n))} for n in range(2, 17)},
    }
    return header, json.dumps(data, indent=1) + "\n"


def generate(check_only: bool = False) -> int:
    chosen = choose_networks()
    for n, rec in chosen.items():
        if not sorts_all_01(n, rec["pairs"]):
            raise RuntimeError(f"network for n={n} does not sort")
    for n in range(2, 17):
        if not sorts_all_01(n, bose_nelson(n)):
            raise RuntimeError(f"Bose-Nelson network for n={n} does not sort")
    masks = warp_schedule(32)
    header, data = render(chosen, masks)
    if check_only:
        stale = []
        for path, text in ((HEADER, header), (JSON_OUT, data)):
            if not os.path.exists(path) or open(path).read() != text:
                stale.append(path)
        if stale:
            print("stale:", *stale)
            return 1
        return 0
    with open(HEADER, "w") as f:
        f.write(header)
    with open(JSON_OUT, "w") as f:
        f.write(data)
    for n in range(2, 17):
        net = chosen[n]["pairs"]
        print(f"n={n:2d} size={len(net):2d} (best known {BEST_KNOWN_SIZE[n]:2d}) "
              f"depth={depth(n, net):2d} from {chosen[n]['provenance']}")
    return 0


def search(n: int, restarts: int, seeds, prefix_levels=None) -> None:
    """Run search.c from prefixes taken from the chosen networks and store any
    improvement in searched.json (with the command that reproduces it)."""
    exe = os.path.join(HERE, "_search")
    src = os.path.join(HERE, "search.c")
    subprocess.check_call(["gcc", "-O2", "-o", exe, src])
    chosen = choose_networks()
    current = chosen[n]["pairs"]
    best = len(current)
    found = None
    levels = prefix_levels if prefix_levels else [1, 2, 3]
    for L in levels:
        # prefix: the comparators of the current network in its first L levels
        last = [0] * n
        prefix = []
        for i, j in current:
            lv = max(last[i], last[j]) + 1
            last[i] = last[j] = lv
            if lv <= L:
                prefix.append((i, j))
        for seed in seeds:
            args = [exe, str(n), str(restarts), str(seed)] + [str(x) for p in prefix for x in p]
            out = subprocess.run(args, capture_output=True, text=True).stdout.split("\n")
            if not out[0].startswith("size ") or out[0] == "size none":
                continue
            size = int(out[0].split()[1])
            pairs = [tuple(int(x) for x in ln.split()) for ln in out[1:] if ln.strip()]
            print(f"n={n} L={L} seed={seed}: {size}", flush=True)
            if size < best and sorts_all_01(n, pairs):
                best = size
                found = {"n": n, "pairs": [list(p) for p in pairs],
                         "provenance": f"search(prefix=levels<={L} of the chosen n={n} network, "
                                       f"restarts={restarts}, seed={seed})"}
    if found:
        recs = json.load(open(SEARCHED)) if os.path.exists(SEARCHED) else []
        recs = [r for r in recs if r["n"] != n] + [found]
        with open(SEARCHED, "w") as f:
            json.dump(recs, f, indent=1)
            f.write("\n")
        print("improved:", found["provenance"], best)


def evolve(n: int, target: int, seed: int, seconds: float, reflection: bool, prefix, env=None) -> bool:
    """Run evolve.c (deterministic for a seed: it stops at the target size) and
    store a network smaller than the chosen one in searched.json."""
    exe = os.path.join(HERE, "_evolve")
    subprocess.check_call(["gcc", "-O3", "-o", exe, os.path.join(HERE, "evolve.c")])
    args = [exe, str(n), str(target), str(seed), str(seconds), "1" if reflection else "0"]
    args += [str(x) for p in prefix for x in p]
    run_env = dict(os.environ, **{k: str(v) for k, v in (env or {}).items()})
    out = subprocess.run(args, capture_output=True, text=True, env=run_env).stdout.split("\n")
    heads = [k for k, ln in enumerate(out) if ln.startswith("size ")]
    if not heads:
        return False
    size = int(out[heads[-1]].split()[1])
    pairs = [tuple(int(x) for x in ln.split()) for ln in out[heads[-1] + 1:heads[-1] + 1 + size]]
    if size >= len(choose_networks()[n]["pairs"]) or not sorts_all_01(n, pairs):
        return False
    knobs = ", ".join(f"{k}={v}" for k, v in (env or {}).items())
    pre = "".join(f"({i},{j})" for i, j in prefix)
    recs = [r for r in _searched() if r["n"] != n]
    recs.append({"n": n, "pairs": [list(p) for p in pairs],
                 "provenance": f"evolve(n={n}, target={target}, seed={seed}"
                               f"{', reflection' if reflection else ''}, prefix={pre}{', ' + knobs if knobs else ''})"})
    with open(SEARCHED, "w") as f:
        json.dump(recs, f, indent=1)
        f.write("\n")
    print(f"n={n}: {size} comparators from evolve.c")
    return True


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--check", action="store_true", help="fail if the outputs are stale")
    ap.add_argument("--search", type=int, default=0, help="search for a smaller network for N")
    ap.add_argument("--restarts", type=int, default=200)
    ap.add_argument("--seeds", type=int, nargs="*", default=[1, 2, 3])
    ap.add_argument("--levels", type=int, nargs="*", default=None)
    ap.add_argument("--evolve13", action="store_true",
                    help="rerun the evolutionary search that found the 45-comparator n=13 network")
    args = ap.parse_args(argv)
    if args.evolve13:
        evolve(13, 45, 35, 3600, True, [(0, 1), (2, 3), (4, 5), (7, 8), (9, 10), (11, 12)],
               {"EVOLVE_RANDOM": 40, "EVOLVE_WORSE": 20})
        return 0
    if args.search:
        search(args.search, args.restarts, args.seeds, args.levels)
        return 0
    return generate(check_only=args.check)


if __name__ == "__main__":
    sys.exit(main())
