"""Pins for the CPU oracle: checks against facts the paper and mathematics fix,
independent of the oracle's own code.

* sorting: brute force over all permutations (output must be 0..n-1), numpy's
  stable sort (a library routine the definition reduces to), the sorted +
  permutation invariants of Sec. 4.1;
* networks: the paper's printed networks (tests/golden) must pass, their stated
  sizes and depths must be reproduced, and dropping any comparator from a
  size-optimal network must make it fail;
* mutation tests compile deliberately broken copies of oracle.c and check that
  these pins catch each mistake.
"""
import ctypes
import itertools
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle import rss
from paper_2002_05599_gb300 import workloads as wl


# ---------------------------------------------------------------- sorting ----

@pytest.mark.parametrize("n", range(2, 8))
def test_sort_fixed_all_permutations(n):
    perms = np.array(list(itertools.permutations(range(n))), dtype=np.uint32)
    out = oracle.sort_fixed(perms.reshape(-1), n).reshape(-1, n)
    assert (out == np.arange(n, dtype=np.uint32)).all()


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("dist", ["uniform", "fewdistinct", "presorted", "reverse"])
def test_sort_fixed_matches_numpy(dtype, dist):
    for n in range(2, 17):
        keys = wl.fixed_arrays(n, 257, dist, dtype, seed=3 + n)
        out = oracle.sort_fixed(keys, n)
        ref = np.sort(keys.reshape(-1, n), axis=1).reshape(-1)
        assert np.array_equal(out, ref)


def _stable_reference(keys, vals, offsets):
    k = keys.copy()
    v = None if vals is None else vals.copy()
    for s in range(offsets.size - 1):
        a, b = int(offsets[s]), int(offsets[s + 1])
        order = np.argsort(keys[a:b], kind="stable")
        k[a:b] = keys[a:b][order]
        if v is not None:
            v[a:b] = vals[a:b][order]
    return k, v


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("keys", ["uniform", "fewdistinct", "zipf"])
def test_sort_segments_matches_numpy_stable(dtype, keys):
    k, v, off = wl.segment_batch(400, "geometric", keys, dtype, True, seed=7)
    got_k, got_v = oracle.sort_segments(k, v, off)
    ref_k, ref_v = _stable_reference(k, v, off)
    assert np.array_equal(got_k, ref_k)
    assert np.array_equal(got_v, ref_v)


def test_sort_segments_edge_cases():
    # empty, length-1, all-equal, max-key and a non-zero first offset;
    # elements outside the segments must stay untouched
    keys = np.array([9, 9, 5, 5, 5, 0xFFFFFFFF, 3, 0xFFFFFFFF, 1, 7, 7], dtype=np.uint32)
    vals = np.arange(keys.size, dtype=np.uint32) + 100
    off = np.array([2, 2, 3, 5, 8, 8, 10], dtype=np.uint32)
    got_k, got_v = oracle.sort_segments(keys, vals, off)
    assert got_k.tolist() == [9, 9, 5, 5, 5, 3, 0xFFFFFFFF, 0xFFFFFFFF, 1, 7, 7]
    assert got_v.tolist() == [100, 101, 102, 103, 104, 106, 105, 107, 108, 109, 110]


def test_sort_segments_stability_brute_force():
    # all 3^5 sequences over {0,1,2}: output order = (key, original position)
    seqs = np.array(list(itertools.product(range(3), repeat=5)), dtype=np.uint64)
    off = np.arange(0, seqs.size + 1, 5, dtype=np.uint32)
    vals = np.tile(np.arange(5, dtype=np.uint32), len(seqs))
    k, v = oracle.sort_segments(seqs.reshape(-1), vals, off)
    for s, seq in enumerate(seqs.tolist()):
        expect = sorted(range(5), key=lambda i: (seq[i], i))
        assert v[5 * s:5 * s + 5].tolist() == expect
        assert k[5 * s:5 * s + 5].tolist() == [seq[i] for i in expect]


def test_perm_product_definition_and_invariants():
    rng = np.random.default_rng(5)
    a = rng.integers(0, 2**63, size=300, dtype=np.uint64)
    p, z = oracle.PERM_P, oracle.PERM_Z
    expect = 1
    for x in a.tolist():
        expect = expect * ((z - x) % p) % p
    assert oracle.perm_product(a, z, p) == expect
    assert oracle.perm_product(rng.permutation(a), z, p) == expect
    b = a.copy()
    b[17] = b[18]  # a planted duplication must change v
    assert oracle.perm_product(b, z, p) != expect
    a32 = a.astype(np.uint32)
    assert oracle.perm_product(a32, z, p) == oracle.perm_product(a32.astype(np.uint64), z, p)
    # z is bumped until v != 0 (Sec. 4.1)
    c = np.array([oracle.PERM_Z, 1, 2], dtype=np.uint64)
    assert oracle.perm_product(c) == 0
    assert oracle.perm_check_z(c) == oracle.PERM_Z + 1


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_is_sorted_segments(dtype):
    # Sec. 4.1's sorted check, per segment: a descent across a segment
    # boundary or inside an empty segment's neighbourhood is allowed, equal
    # neighbours are sorted, any descent inside a segment is not
    off = np.array([0, 3, 3, 5], dtype=np.uint32)
    assert oracle.is_sorted_segments(np.array([1, 2, 2, 0, 9], dtype=dtype), off)
    assert not oracle.is_sorted_segments(np.array([1, 2, 2, 9, 8], dtype=dtype), off)
    assert not oracle.is_sorted_segments(np.array([2, 1, 2, 0, 9], dtype=dtype), off)  # first pair
    top = np.iinfo(dtype).max
    assert oracle.is_sorted_segments(np.array([top, top, top], dtype=dtype), np.array([0, 3], np.uint32))
    assert not oracle.is_sorted_segments(np.array([top, 0], dtype=dtype), np.array([0, 2], np.uint32))
    # against a direct Python check on random batches with a few planted descents
    rng = np.random.default_rng(17)
    k, _, off = wl.segment_batch(300, "geometric", "fewdistinct", dtype, False, seed=18)
    srt, _ = oracle.sort_segments(k, None, off)
    assert oracle.is_sorted_segments(srt, off)
    for _ in range(30):
        bad = srt.copy()
        i = int(rng.integers(1, bad.size))
        bad[i - 1], bad[i] = bad[i], bad[i - 1]
        expect = all(bad[e - 1] <= bad[e] for s in range(off.size - 1)
                     for e in range(int(off[s]) + 1, int(off[s + 1])))
        assert oracle.is_sorted_segments(bad, off) == expect


# --------------------------------------------------------------- networks ----

@pytest.mark.parametrize("name", ["best16", "opt10", "bn6", "bnl16", "bnp16"])
def test_printed_networks_sort(golden_networks, name):
    n, facts, levels = golden_networks[name]
    pairs = [p for lv in levels for p in lv]
    assert len(pairs) == facts["size"]
    assert oracle.network_failures_01(n, pairs) == 0


@pytest.mark.parametrize("name", ["best16", "opt10"])
def test_printed_levels_and_depth(golden_networks, name):
    n, facts, levels = golden_networks[name]
    assert len(levels) == facts["levels"]
    for lv in levels:  # a level's comparators share no channel (Sec. 2.1)
        chans = [c for p in lv for c in p]
        assert len(chans) == len(set(chans))
    pairs = [p for lv in levels for p in lv]
    assert oracle.network_depth(n, pairs) == facts["levels"]


def test_depth_small_cases():
    assert oracle.network_depth(2, [(0, 1)]) == 1
    assert oracle.network_depth(4, [(0, 1), (2, 3)]) == 1
    assert oracle.network_depth(3, [(0, 1), (1, 2), (0, 1)]) == 3
    assert oracle.network_depth(4, [(0, 1), (2, 3), (0, 2), (1, 3), (1, 2)]) == 3


@pytest.mark.parametrize("name", ["best16", "opt10"])
def test_dropping_any_comparator_breaks_best_networks(golden_networks, name):
    # 29 is the optimal size for n=10 (Sec. 2.1) and 60 the best known for n=16:
    # no sorting network with one comparator fewer can exist / is known.
    n, _, levels = golden_networks[name]
    pairs = [p for lv in levels for p in lv]
    for c in range(len(pairs)):
        assert oracle.network_failures_01(n, pairs[:c] + pairs[c + 1:]) > 0


def test_perm_and_01_checkers_agree(golden_networks):
    n, _, levels = golden_networks["opt10"]
    pairs = [p for lv in levels for p in lv]
    assert oracle.network_failures_perm(n, pairs) == 0
    assert oracle.network_failures_perm(n, pairs[:-1]) > 0
    n6, _, lv6 = golden_networks["bn6"]
    p6 = [p for lv in lv6 for p in lv]
    for c in range(len(p6)):
        broken = p6[:c] + p6[c + 1:]
        assert (oracle.network_failures_perm(n6, broken) > 0) == \
               (oracle.network_failures_01(n6, broken) > 0)


def _perm_failures_python(n, pairs):
    fails = 0
    for p in itertools.permutations(range(n)):
        x = list(p)
        for i, j in pairs:
            if x[i] > x[j]:
                x[i], x[j] = x[j], x[i]
        fails += x != sorted(x)
    return fails


def test_perm_checker_counts_like_brute_force(golden_networks):
    n6, _, lv6 = golden_networks["bn6"]
    p6 = [p for lv in lv6 for p in lv]
    for c in (0, 5, len(p6) - 1):
        broken = p6[:c] + p6[c + 1:]
        assert oracle.network_failures_perm(n6, broken) == _perm_failures_python(n6, broken)


def test_wide_01_checker_matches_plain(golden_networks):
    rng = np.random.default_rng(11)
    for name in ["best16", "opt10", "bnl16"]:
        n, _, levels = golden_networks[name]
        pairs = [p for lv in levels for p in lv]
        for trial in range(4):
            net = list(pairs)
            if trial:
                del net[int(rng.integers(len(net)))]
            assert oracle.network_failures_01_wide(n, net) == oracle.network_failures_01(n, net)


def test_insertion_network_brute_force():
    # the "bubble" network of Knuth 5.3.4 sorts; its count of 0-1 failures after
    # removing the last comparator equals a direct count
    n = 6
    pairs = [(j, j + 1) for i in range(n - 1, 0, -1) for j in range(i)]
    assert oracle.network_failures_01(n, pairs) == 0
    broken = pairs[:-1]
    direct = 0
    for v in range(1 << n):
        x = [(v >> i) & 1 for i in range(n)]
        for i, j in broken:
            if x[i] > x[j]:
                x[i], x[j] = x[j], x[i]
        direct += any(x[i] > x[i + 1] for i in range(n - 1))
    assert oracle.network_failures_01(n, broken) == direct


# -------------------------------------------------------------------- RSS ----

def test_rss_tree_classification_matches_definition():
    rng = np.random.default_rng(2)
    for k in (2, 4, 8, 16, 32):
        spl = sorted(rng.choice(1000, size=k - 1, replace=False).tolist())
        tree = rss.heap_tree(spl)
        assert tree[1] == spl[k // 2 - 1]  # root is s_(k/2)
        for e in range(-2, 1003):
            assert rss.classify_tree(e, tree) == rss.classify_definition(e, spl)


@pytest.mark.parametrize("k,a", [(4, 3), (4, 1), (8, 2), (16, 2), (32, 3)])
def test_rss_sorts(k, a):
    rng = np.random.default_rng(k * 10 + a)
    for length in (17, 33, 100, 256):
        keys = rng.integers(0, 5, size=length).tolist()  # heavy duplicates
        items = [(x, i) for i, x in enumerate(keys)]
        assert rss.rss_sort(items, k, a) == sorted(items)


# --------------------------------------------------------------- mutation ----

def _random_items(count, n, seed):
    """Interleaved (key, ref) items with many equal keys; ref = input position."""
    rng = np.random.default_rng(seed)
    items = np.empty(2 * count * n, np.uint64)
    items[0::2] = rng.integers(0, 5, count * n, dtype=np.uint64)
    items[1::2] = np.arange(count * n, dtype=np.uint64)
    return items


def _items_reference(items, n):
    """Each array ordered by (key, position in the array): Python's sort of index tuples."""
    out = items.copy().reshape(-1, n, 2)
    for a in range(out.shape[0]):
        rows = [(int(out[a, i, 0]), i, int(out[a, i, 1])) for i in range(n)]
        rows.sort()
        for i, (k, _, r) in enumerate(rows):
            out[a, i, 0], out[a, i, 1] = k, r
    return out.reshape(-1)


def test_array_merge_sort_matches_numpy_and_insertion_sort():
    for n in (0, 1, 2, 3, 7, 64, 1000, 4097, 100_003):
        keys = wl.uniform_keys(n, np.uint32, n + 1) % np.uint32(max(1, n // 3))
        got = oracle.sort_array(keys)
        assert np.array_equal(got, np.sort(keys))
        if 0 < n <= 4097:  # the same result as the insertion-sort oracle on one array
            assert np.array_equal(got, oracle.sort_fixed(keys, n))


def test_items_sort_is_stable_by_key_with_references_attached():
    for n in (2, 3, 8, 16):
        items = _random_items(200, n, seed=n)
        got = oracle.sort_fixed_items(items, n)
        assert np.array_equal(got, _items_reference(items, n))
        # keys alone agree with the keys-only oracle and numpy
        keys = items[0::2].copy()
        assert np.array_equal(got[0::2], oracle.sort_fixed(keys, n))
        assert np.array_equal(got[0::2], np.sort(keys.reshape(-1, n), axis=1).reshape(-1))
        # every (key, ref) pair survives
        pairs_in = sorted(zip(items[0::2].tolist(), items[1::2].tolist()))
        pairs_out = sorted(zip(got[0::2].tolist(), got[1::2].tolist()))
        assert pairs_in == pairs_out


def _f32(bits):
    return np.array(bits, dtype=np.uint32).view(np.float32)


def _total_order_key32(bits):
    """IEEE 754 totalOrder of a binary32 bit pattern as a Python sort key, from
    the standard's cases (NaN class by sign, numbers by value, -0 before +0,
    NaNs of one sign by payload)."""
    import math
    bits = int(bits)
    x = float(np.array([bits], np.uint32).view(np.float32)[0])  # numeric value (exact for non-NaN)
    payload = bits & 0x7FFFFFFF
    if (bits >> 23) & 0xFF == 0xFF and bits & 0x7FFFFF:  # NaN, read from the bits
        return (0, -payload) if bits >> 31 else (2, payload)
    zero_rank = 0 if math.copysign(1.0, x) < 0 else 1
    return (1, x, zero_rank)


def test_float_keys_follow_total_order_on_special_values():
    expect = _f32([0xFFFFFFFF, 0xFFC00001, 0xFF800000, 0xFF7FFFFF, 0xBF800000, 0x80000001, 0x80000000,
                   0x00000000, 0x00000001, 0x3F800000, 0x7F7FFFFF, 0x7F800000, 0x7F800001, 0x7FC00000,
                   0x7FFFFFFF])
    rng = np.random.default_rng(3)
    for _ in range(20):
        shuffled = rng.permutation(expect)
        got = oracle.sort_fixed(shuffled, expect.size)
        assert np.array_equal(got.view(np.uint32), expect.view(np.uint32))


def test_float_keys_match_numpy_on_ordinary_values():
    rng = np.random.default_rng(4)
    for dt in (np.float32, np.float64):
        keys = (rng.standard_normal(16 * 500) * 1e3).astype(dt)
        keys[keys == 0] = 1  # no signed zeros: numpy treats -0 == +0
        assert np.array_equal(oracle.sort_fixed(keys, 16), np.sort(keys.reshape(-1, 16), 1).reshape(-1))


def test_float_keys_on_random_bit_patterns_against_python():
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 2**32, 8 * 2000, dtype=np.uint64).astype(np.uint32)
    bits[::7] = rng.choice([0x7FC00000, 0xFFC00000, 0x80000000, 0, 0x7F800000, 0xFF800000], bits[::7].size)
    keys = bits.view(np.float32)
    got = oracle.sort_fixed(keys, 8).view(np.uint32).reshape(-1, 8)
    for a, row in enumerate(bits.reshape(-1, 8)):
        order = sorted(range(8), key=lambda i: (_total_order_key32(row[i]), i))
        assert np.array_equal(got[a], row[order])
    # segments with payload: stable among equal bit patterns
    k, v, off = wl.segment_batch(300, "geometric", "fewdistinct", np.uint32, True, seed=6)
    kf = k.astype(np.float32) - np.float32(1.5)  # few distinct values, both signs
    kb = kf.view(np.uint32)
    gk, gv = oracle.sort_segments(kf, v, off)
    for sgm in range(off.size - 1):
        lo, hi = int(off[sgm]), int(off[sgm + 1])
        order = sorted(range(lo, hi), key=lambda i: (_total_order_key32(kb[i]), i))
        assert np.array_equal(gk[lo:hi], kf[order]) and np.array_equal(gv[lo:hi], v[order])



def _total_order_key64(bits):
    """IEEE 754 totalOrder of a binary64 bit pattern as a Python sort key, from
    the standard's cases: NaNs (exponent all ones, fraction non-zero) with the
    sign bit set come before everything and order by decreasing payload, those
    without it after everything by increasing payload; other values order by
    numeric value, with -0 before +0."""
    import math
    bits = int(bits)
    if (bits >> 52) & 0x7FF == 0x7FF and bits & ((1 << 52) - 1):
        payload = bits & ((1 << 63) - 1)
        return (0, -payload) if bits >> 63 else (2, payload)
    x = float(np.array([bits], np.uint64).view(np.float64)[0])  # exact for non-NaN
    return (1, x, 0 if math.copysign(1.0, x) < 0 else 1)


# binary64 bit patterns in totalOrder, written out from the standard's cases:
# negative NaNs (largest payload first; quiet and signalling), -inf, negative
# normal and subnormal numbers, -0, +0, positive numbers, +inf, positive NaNs.
_F64_ORDERED = [
    0xFFFFFFFFFFFFFFFF, 0xFFF8000000000001, 0xFFF8000000000000, 0xFFF4000000000000, 0xFFF0000000000001,
    0xFFF0000000000000, 0xFFEFFFFFFFFFFFFF, 0xBFF0000000000000, 0x800FFFFFFFFFFFFF, 0x8000000000000001,
    0x8000000000000000, 0x0000000000000000, 0x0000000000000001, 0x000FFFFFFFFFFFFF, 0x3FF0000000000000,
    0x7FEFFFFFFFFFFFFF, 0x7FF0000000000000, 0x7FF0000000000001, 0x7FF4000000000000, 0x7FF8000000000000,
    0x7FF8000000000001, 0x7FFFFFFFFFFFFFFF,
]


def test_f64_keys_follow_total_order_on_special_values():
    expect = np.array(_F64_ORDERED, np.uint64)
    # the written-out order agrees with the case-by-case key (two independent statements)
    assert sorted(_F64_ORDERED, key=_total_order_key64) == _F64_ORDERED
    rng = np.random.default_rng(13)
    for _ in range(20):
        shuffled = rng.permutation(expect).view(np.float64)
        got = oracle.sort_fixed(shuffled, expect.size)
        assert np.array_equal(got.view(np.uint64), expect)


def _f64_mix(rng, size):
    """binary64 bit patterns from a small pool of special values (both NaN
    signs with several payloads, signed zeros, infinities) and random bits."""
    pool = np.array(_F64_ORDERED, np.uint64)
    bits = rng.integers(0, 2**63, size, dtype=np.uint64) | (rng.integers(0, 2, size, dtype=np.uint64) << np.uint64(63))
    pick = rng.random(size) < 0.6
    bits[pick] = rng.choice(pool, int(pick.sum()))
    return bits


def test_f64_keys_on_random_bit_patterns_against_python():
    rng = np.random.default_rng(14)
    bits = _f64_mix(rng, 8 * 1500)
    got = oracle.sort_fixed(bits.view(np.float64), 8).view(np.uint64).reshape(-1, 8)
    for a, row in enumerate(bits.reshape(-1, 8)):
        order = sorted(range(8), key=lambda i: (_total_order_key64(row[i]), i))
        assert np.array_equal(got[a], row[order])


def test_f64_segments_stable_against_python():
    # oracle_sort_segments_f64: equal bit patterns (many, from the small pool)
    # keep their input order and the payload moves with its key
    rng = np.random.default_rng(15)
    _, v, off = wl.segment_batch(400, "geometric", "uniform", np.uint64, True, seed=16)
    bits = _f64_mix(rng, int(off[-1]))
    gk, gv = oracle.sort_segments(bits.view(np.float64), v, off)
    gk = gk.view(np.uint64)
    for sgm in range(off.size - 1):
        lo, hi = int(off[sgm]), int(off[sgm + 1])
        order = sorted(range(lo, hi), key=lambda i: (_total_order_key64(bits[i]), i))
        assert np.array_equal(gk[lo:hi], bits[order]) and np.array_equal(gv[lo:hi], v[order])
    # keys only (no payload) gives the same keys
    gk2, gv2 = oracle.sort_segments(bits.view(np.float64), None, off)
    assert gv2 is None and np.array_equal(gk2.view(np.uint64), gk)

_MUTATIONS = {
    # a wrong comparison sign in the fixed-size insertion sort
    "fixed_sign": ("while (j >= 0 && A[j] > x) {\n                A[j + 1] = A[j];\n                --j;\n            }\n            A[j + 1] = x;\n        }\n    }\n}\n\nvoid oracle_sort_fixed_u64",
                   "while (j >= 0 && A[j] < x) {\n                A[j + 1] = A[j];\n                --j;\n            }\n            A[j + 1] = x;\n        }\n    }\n}\n\nvoid oracle_sort_fixed_u64"),
    # an unstable segment sort (moves past equal keys)
    "seg_unstable": ("while (j >= 0 && A[j] > x) {\n                A[j + 1] = A[j];\n                if (V) V[j + 1] = V[j];\n                --j;\n            }\n            A[j + 1] = x;\n            if (V) V[j + 1] = v;\n        }\n    }\n}\n\nvoid oracle_sort_segments_u64",
                     "while (j >= 0 && A[j] >= x) {\n                A[j + 1] = A[j];\n                if (V) V[j + 1] = V[j];\n                --j;\n            }\n            A[j + 1] = x;\n            if (V) V[j + 1] = v;\n        }\n    }\n}\n\nvoid oracle_sort_segments_u64"),
    # payload not moved with its key
    "seg_payload": ("if (V) V[j + 1] = V[j];\n                --j;\n            }\n            A[j + 1] = x;\n            if (V) V[j + 1] = v;\n        }\n    }\n}\n\nvoid oracle_sort_segments_u64",
                    "--j;\n            }\n            A[j + 1] = x;\n            if (V) V[j + 1] = v;\n        }\n    }\n}\n\nvoid oracle_sort_segments_u64"),
    # the network comparator exchanges in the wrong direction
    "net_direction": ("if (x[lo[c]] > x[hi[c]]) {", "if (x[lo[c]] < x[hi[c]]) {"),
    # the 0-1 vectors skip the top channel's bit
    "net_index": ("for (int i = 0; i < n; ++i) x[i] = (int64_t)((v >> i) & 1u);",
                  "for (int i = 0; i < n; ++i) x[i] = (int64_t)((v >> i) & 1u) * (i + 1 < n);"),
    # depth forgets the +1 per comparator
    "depth": ("        l += 1;\n", ""),
    # unstable item sort (moves past equal keys)
    "items_unstable": ("while (j >= 0 && A[2 * j] > key) {", "while (j >= 0 && A[2 * j] >= key) {"),
    # the reference is not moved with its key
    "items_ref": ("                A[2 * (j + 1) + 1] = A[2 * j + 1];\n", ""),
    # -0 and +0 in the wrong order
    "float_zero": ("return (signbit(a) == 0) && (signbit(b) != 0); /* +0 after -0 */",
                   "return (signbit(a) != 0) && (signbit(b) == 0); /* +0 after -0 */"),
    # negative NaNs ordered by payload the wrong way
    "float_nan": ("    pa &= 0x7FFFFFFFu;\n    pb &= 0x7FFFFFFFu;\n    return ca > 0 ? pa > pb : pa < pb;",
                  "    pa &= 0x7FFFFFFFu;\n    pb &= 0x7FFFFFFFu;\n    return pa > pb;"),
    # the merge takes from the right run on ties and drops the last element of a run
    "merge_drop": ("while (i < mid) dst[o++] = src[i++];", "while (i + 1 < mid) dst[o++] = src[i++];"),
    # the permutation product drops a term
    "perm": ("    for (uint64_t i = 0; i < len; ++i) {\n        uint64_t ar = a[i] % p;",
             "    for (uint64_t i = 1; i < len; ++i) {\n        uint64_t ar = a[i] % p;"),
    # the u32 permutation product drops its last term
    "perm_u32": ("    for (uint64_t i = 0; i < len; ++i) {\n        uint64_t ar = (uint64_t)a[i] % p;",
                 "    for (uint64_t i = 0; i + 1 < len; ++i) {\n        uint64_t ar = (uint64_t)a[i] % p;"),
    # a wrong comparison sign in the u64 fixed-size sort
    "fixed_u64_sign": ("while (j >= 0 && A[j] > x) {\n                A[j + 1] = A[j];\n                --j;\n            }\n            A[j + 1] = x;\n        }\n    }\n}\n\n/*\n * The 16-byte items",
                       "while (j >= 0 && A[j] < x) {\n                A[j + 1] = A[j];\n                --j;\n            }\n            A[j + 1] = x;\n        }\n    }\n}\n\n/*\n * The 16-byte items"),
    # an unstable u64 segment sort
    "seg_u64_unstable": ("while (j >= 0 && A[j] > x) {\n                A[j + 1] = A[j];\n                if (V) V[j + 1] = V[j];\n                --j;\n            }\n            A[j + 1] = x;\n            if (V) V[j + 1] = v;\n        }\n    }\n}\n\n/*\n * One array",
                         "while (j >= 0 && A[j] >= x) {\n                A[j + 1] = A[j];\n                if (V) V[j + 1] = V[j];\n                --j;\n            }\n            A[j + 1] = x;\n            if (V) V[j + 1] = v;\n        }\n    }\n}\n\n/*\n * One array"),
    # f32: -0 and +0 in the wrong order
    "f32_zero": ("        return (signbit(a) == 0) && (signbit(b) != 0);\n    }\n    uint32_t pa, pb;",
                 "        return (signbit(a) != 0) && (signbit(b) == 0);\n    }\n    uint32_t pa, pb;"),
    # f64: negative NaNs ordered by payload the wrong way (as if positive)
    "f64_nan_payload": ("    pa &= 0x7FFFFFFFFFFFFFFFull;\n    pb &= 0x7FFFFFFFFFFFFFFFull;\n    return ca > 0 ? pa > pb : pa < pb;",
                        "    pa &= 0x7FFFFFFFFFFFFFFFull;\n    pb &= 0x7FFFFFFFFFFFFFFFull;\n    return pa > pb;"),
    # f64: the NaN classes in the wrong order (negative NaNs last)
    "f64_nan_class": ("    if (ca != cb) return ca > cb;\n    if (ca == 0) {\n        if (a != b) return a > b;\n        return (signbit(a) == 0) && (signbit(b) != 0); /* +0 after -0 */",
                      "    if (ca != cb) return ca < cb;\n    if (ca == 0) {\n        if (a != b) return a > b;\n        return (signbit(a) == 0) && (signbit(b) != 0); /* +0 after -0 */"),
    # f64 segments: the payload is not moved with its key
    "seg_f64_payload": ("            while (j >= 0 && greater_f64(A[j], x)) {\n                A[j + 1] = A[j];\n                if (V) V[j + 1] = V[j];",
                        "            while (j >= 0 && greater_f64(A[j], x)) {\n                A[j + 1] = A[j];"),
    # the u32 sorted check skips the first pair of every segment
    "sorted_u32": ("int oracle_is_sorted_segments_u32(const uint32_t *keys, const uint32_t *offsets, uint64_t nseg)\n{\n    for (uint64_t s = 0; s < nseg; ++s)\n        for (uint64_t i = (uint64_t)offsets[s] + 1;",
                   "int oracle_is_sorted_segments_u32(const uint32_t *keys, const uint32_t *offsets, uint64_t nseg)\n{\n    for (uint64_t s = 0; s < nseg; ++s)\n        for (uint64_t i = (uint64_t)offsets[s] + 2;"),
    # the u64 sorted check rejects equal neighbours
    "sorted_u64": ("            if (keys[i - 1] > keys[i]) return 0;\n    return 1;\n}\n\nint oracle_is_sorted_segments_u32",
                   "            if (keys[i - 1] >= keys[i]) return 0;\n    return 1;\n}\n\nint oracle_is_sorted_segments_u32"),
    # the permutation checker feeds values with pairs made equal
    "perm_values": ("        for (int i = 0; i < n; ++i) x[i] = p[i];\n", "        for (int i = 0; i < n; ++i) x[i] = p[i] / 2;\n"),
    # the wide 0-1 checker gives channels 0 and 1 the same input bits
    "wide_pattern": ("0xAAAAAAAAAAAAAAAAull, 0xCCCCCCCCCCCCCCCCull,", "0xAAAAAAAAAAAAAAAAull, 0xAAAAAAAAAAAAAAAAull,"),
}


def _pins_pass(lib_path, golden):
    """Run a compact version of the pins above against a given oracle build."""
    saved = oracle._lib
    try:
        oracle._lib = None
        lib = ctypes.CDLL(lib_path)
        oracle._lib = None
        # reuse the argtype setup of the real loader
        real = oracle._LIB_PATH
        oracle._LIB_PATH = lib_path
        oracle._lib = None
        try:
            oracle._load()
        finally:
            oracle._LIB_PATH = real
        ok = True
        keys = wl.fixed_arrays(8, 64, "uniform", np.uint32, seed=9)
        ok &= np.array_equal(oracle.sort_fixed(keys, 8), np.sort(keys.reshape(-1, 8), 1).reshape(-1))
        for dt in (np.uint32, np.uint64):
            k, v, off = wl.segment_batch(200, "geometric", "fewdistinct", dt, True, seed=9)
            gk, gv = oracle.sort_segments(k, v, off)
            rk, rv = _stable_reference(k, v, off)
            ok &= np.array_equal(gk, rk) and np.array_equal(gv, rv)
        special = _f32([0xFFC00000, 0xFFC00001, 0x80000000, 0, 0x7FC00001, 0x7FC00000, 0xBF800000])
        ok &= np.array_equal(oracle.sort_fixed(special, 7).view(np.uint32),
                             np.array([0xFFC00001, 0xFFC00000, 0xBF800000, 0x80000000, 0, 0x7FC00000,
                                       0x7FC00001], np.uint32))
        special64 = np.array([0x8000000000000000, 0, 0xBFF0000000000000, 0x7FF8000000000000], np.uint64)
        ok &= np.array_equal(oracle.sort_fixed(special64[[1, 3, 0, 2]].view(np.float64), 4).view(np.uint64),
                             special64[[2, 0, 1, 3]])
        keys64 = wl.fixed_arrays(8, 64, "uniform", np.uint64, seed=9)
        ok &= np.array_equal(oracle.sort_fixed(keys64, 8), np.sort(keys64.reshape(-1, 8), 1).reshape(-1))
        f64 = np.array(_F64_ORDERED, np.uint64)
        got = oracle.sort_fixed(np.random.default_rng(9).permutation(f64).view(np.float64), f64.size)
        ok &= np.array_equal(got.view(np.uint64), f64)
        rng = np.random.default_rng(10)
        _, v, off = wl.segment_batch(60, "geometric", "uniform", np.uint64, True, seed=10)
        bits = _f64_mix(rng, int(off[-1]))
        gk, gv = oracle.sort_segments(bits.view(np.float64), v, off)
        for sgm in range(off.size - 1):
            lo, hi = int(off[sgm]), int(off[sgm + 1])
            order = sorted(range(lo, hi), key=lambda i: (_total_order_key64(bits[i]), i))
            ok &= np.array_equal(gk.view(np.uint64)[lo:hi], bits[order]) and np.array_equal(gv[lo:hi], v[order])
        for dt in (np.uint32, np.uint64):
            soff = np.array([0, 3, 3, 5], dtype=np.uint32)
            ok &= oracle.is_sorted_segments(np.array([1, 2, 2, 0, 9], dtype=dt), soff)
            ok &= not oracle.is_sorted_segments(np.array([2, 1, 2, 0, 9], dtype=dt), soff)
        a32 = np.arange(1, 40, dtype=np.uint32)
        expect32 = 1
        for x in a32.tolist():
            expect32 = expect32 * ((oracle.PERM_Z - x) % oracle.PERM_P) % oracle.PERM_P
        ok &= oracle.perm_product(a32) == expect32
        n6, _, lv6 = golden["bn6"]
        p6 = [p for lv in lv6 for p in lv]
        ok &= oracle.network_failures_perm(n6, p6[:-1]) == _perm_failures_python(n6, p6[:-1])
        items = _random_items(40, 7, seed=9)
        ok &= np.array_equal(oracle.sort_fixed_items(items, 7), _items_reference(items, 7))
        arr = wl.uniform_keys(3001, np.uint32, 9) % np.uint32(500)
        ok &= np.array_equal(oracle.sort_array(arr), np.sort(arr))
        n, facts, levels = golden["opt10"]
        pairs = [p for lv in levels for p in lv]
        ok &= oracle.network_failures_01(n, pairs) == 0
        for c in range(len(pairs)):
            broken = pairs[:c] + pairs[c + 1:]
            f = oracle.network_failures_01(n, broken)
            ok &= f > 0 and f == oracle.network_failures_01_wide(n, broken)
        ok &= oracle.network_depth(n, pairs) == facts["levels"]
        a = np.arange(1, 50, dtype=np.uint64)
        expect = 1
        for x in a.tolist():
            expect = expect * ((oracle.PERM_Z - x) % oracle.PERM_P) % oracle.PERM_P
        ok &= oracle.perm_product(a) == expect
        del lib
        return bool(ok)
    finally:
        oracle._lib = saved


def test_pins_pass_on_real_oracle(golden_networks):
    assert _pins_pass(oracle.build(), golden_networks)


@pytest.mark.parametrize("name", sorted(_MUTATIONS))
def test_planted_mistake_is_caught(golden_networks, name):
    src = open(oracle._SRC).read()
    old, new = _MUTATIONS[name]
    assert src.count(old) == 1, "mutation anchor not found"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "m.c")
        so = os.path.join(d, f"libm_{name}.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", so, c])
        assert not _pins_pass(so, golden_networks)
