"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws numbers; it contains no sorting arithmetic, so the CUDA
path and the CPU oracle can both consume its output.  Everything is derived
from SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): output i of the stream with seed s is
``mix(s + (i + 1) * 0x9E3779B97F4A7C15)`` with the published finaliser
``z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
z ^= z >> 31``.  It is counter-based, so any slice can be regenerated alone.

Workloads (the paper measures uniformly random keys, Sec. 4.1, and lists
sorted / reverse inputs as future work):
* fixed-size arrays of u32 / u64 keys: uniform, few-distinct (uniform mod 4),
  presorted and reverse-sorted.  Presorted arrays are built ascending by
  construction (running sums of bounded random increments), reverse ones are
  the same runs read backwards, so no sort is needed to make them;
* CSR segment batches: lengths uniform in [lo, hi] or geometric(p) capped;
  keys uniform or Zipf(s) over ``m`` values; payload = original global index.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream tags so that different quantities drawn from one seed are independent.
TAG_KEYS = 0x6B657973
TAG_LENGTHS = 0x6C656E73
TAG_ZIPF = 0x7A697066


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, tag: int) -> int:
    """Seed of an independent sub-stream: one SplitMix64 output of seed ^ tag."""
    s = np.array([(seed ^ (tag << 20)) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(_mix(s + _GOLDEN)[0])


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream with this seed."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
    return _mix(z)


def _u01(bits: np.ndarray) -> np.ndarray:
    """Map 64 random bits to a double in (0, 1]."""
    return ((bits >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def uniform_keys(count: int, dtype, seed: int = 1, start: int = 0) -> np.ndarray:
    """Keys uniform over the whole range of u32 (top 32 bits) or u64."""
    bits = splitmix64(stream_seed(seed, TAG_KEYS), start, count)
    if np.dtype(dtype) == np.uint32:
        return (bits >> np.uint64(32)).astype(np.uint32)
    return bits


def fixed_arrays(n: int, count: int, dist: str = "uniform", dtype=np.uint32,
                 seed: int = 1) -> np.ndarray:
    """``count`` contiguous arrays of ``n`` keys, flattened (ArrayInRow layout).

    dist: 'uniform' | 'fewdistinct' (uniform mod 4) | 'presorted' | 'reverse'.
    """
    dtype = np.dtype(dtype)
    total = n * count
    if dist == "uniform":
        return uniform_keys(total, dtype, seed)
    if dist == "fewdistinct":
        return uniform_keys(total, dtype, seed) % dtype.type(4)
    if dist in ("presorted", "reverse"):
        top = np.iinfo(dtype).max
        step_max = top // max(n, 1)  # n increments of <= step_max never exceed top
        inc = uniform_keys(total, np.uint64, seed) % np.uint64(step_max + 1)
        runs = np.cumsum(inc.reshape(count, n), axis=1, dtype=np.uint64)
        if dist == "reverse":
            runs = runs[:, ::-1]
        return np.ascontiguousarray(runs).astype(dtype).reshape(-1)
    raise ValueError(f"unknown distribution {dist!r}")


def segment_lengths(nseg: int, kind: str, seed: int = 1, lo: int = 1, hi: int = 16,
                    p: float = 0.15, cap: int = 256) -> np.ndarray:
    """Segment lengths: 'uniform' in [lo, hi] or 'geometric' (success prob p on
    {1, 2, ...}, capped at ``cap``)."""
    bits = splitmix64(stream_seed(seed, TAG_LENGTHS), 0, nseg)
    if kind == "uniform":
        span = np.uint64(hi - lo + 1)
        return (np.uint64(lo) + bits % span).astype(np.uint32)
    if kind == "geometric":
        u = _u01(bits)
        lengths = 1 + np.floor(np.log(u) / np.log1p(-p))
        return np.minimum(lengths, cap).astype(np.uint32)
    raise ValueError(f"unknown length distribution {kind!r}")


def offsets_from_lengths(lengths: np.ndarray) -> np.ndarray:
    """CSR offsets (nseg + 1 entries, first 0) for the given segment lengths."""
    off = np.zeros(lengths.size + 1, dtype=np.uint64)
    np.cumsum(lengths, dtype=np.uint64, out=off[1:])
    if off[-1] >= 2**32:
        raise ValueError("total length must stay below 2^32")
    return off.astype(np.uint32)


def zipf_keys(count: int, s: float = 1.1, m: int = 1 << 20, dtype=np.uint32,
              seed: int = 1) -> np.ndarray:
    """Keys r-1 where rank r in [1, m] has probability proportional to r^-s
    (inverse-CDF sampling)."""
    ranks = np.arange(1, m + 1, dtype=np.float64)
    cdf = np.cumsum(ranks ** (-s))
    u = _u01(splitmix64(stream_seed(seed, TAG_ZIPF), 0, count)) * cdf[-1]
    r = np.searchsorted(cdf, u, side="left")
    r = np.minimum(r, m - 1)
    return r.astype(np.dtype(dtype))


def segment_batch(nseg: int, lengths: str = "uniform", keys: str = "uniform",
                  key_dtype=np.uint64, with_vals: bool = True, seed: int = 1,
                  lo: int = 1, hi: int = 16, p: float = 0.15, cap: int = 256):
    """(keys, vals, offsets) for a CSR batch; vals[i] = i (original global index)."""
    lens = segment_lengths(nseg, lengths, seed, lo=lo, hi=hi, p=p, cap=cap)
    off = offsets_from_lengths(lens)
    total = int(off[-1])
    if keys == "uniform":
        k = uniform_keys(total, key_dtype, seed)
    elif keys == "zipf":
        k = zipf_keys(total, dtype=key_dtype, seed=seed)
    elif keys == "fewdistinct":
        k = uniform_keys(total, key_dtype, seed) % np.dtype(key_dtype).type(4)
    else:
        raise ValueError(f"unknown key distribution {keys!r}")
    v = np.arange(total, dtype=np.uint32) if with_vals else None
    return k, v, off


# ----------------------------------------------------------------------------
# The same SplitMix64 stream evaluated with torch int64 ops on a device, for
# full-size benchmark inputs.  Two's-complement int64 arithmetic wraps like
# u64; right shifts are made logical by masking.

def _as_i64(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


def _lsr(x, s: int):
    return (x >> s) & ((1 << (64 - s)) - 1)


def _mix_torch(z):
    z = (z ^ _lsr(z, 30)) * _as_i64(0xBF58476D1CE4E5B9)
    z = (z ^ _lsr(z, 27)) * _as_i64(0x94D049BB133111EB)
    return z ^ _lsr(z, 31)


def splitmix64_torch(seed: int, start: int, count: int, device):
    """Outputs start .. start+count-1 of the SplitMix64 stream as int64 (same bits as splitmix64)."""
    import torch
    idx = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = _as_i64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _as_i64(0x9E3779B97F4A7C15)
    return _mix_torch(z)


def uniform_keys_torch(count: int, dtype, seed: int = 1, start: int = 0, device="cuda"):
    """uniform_keys on a device: int32 (bits of u32) or int64 (bits of u64) tensor."""
    import torch
    bits = splitmix64_torch(stream_seed(seed, TAG_KEYS), start, count, device)
    if np.dtype(dtype) == np.uint32:
        return _lsr(bits, 32).to(torch.int32)
    return bits


def zipf_keys_torch(count: int, s: float = 1.1, m: int = 1 << 20, dtype=np.uint32, seed: int = 1, device="cuda"):
    """zipf_keys on a device (same values): the CDF is built on the host exactly
    as zipf_keys does, the uniforms come from the same SplitMix64 stream, and
    the inverse-CDF lookup is an exact binary search, so every key matches."""
    import torch
    ranks = np.arange(1, m + 1, dtype=np.float64)
    cdf = torch.from_numpy(np.cumsum(ranks ** (-s))).to(device)
    bits = splitmix64_torch(stream_seed(seed, TAG_ZIPF), 0, count, device)
    u = (_lsr(bits, 11).to(torch.float64) + 1.0) * (1.0 / 9007199254740992.0) * cdf[-1]
    r = torch.clamp(torch.searchsorted(cdf, u, side="left"), max=m - 1)
    return r.to(torch.int32 if np.dtype(dtype) == np.uint32 else torch.int64)
