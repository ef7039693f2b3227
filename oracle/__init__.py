"""Plain CPU oracle for batched small-set sorting (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
and reference arms import this package.  It shares no code with the CUDA
library: ``oracle.c`` is compiled by gcc into ``liboracle.so`` and called
through ctypes on numpy arrays.

Paper: Bingmann, Marianczuk, Sanders, "Engineering Faster Sorters for Small
Sets of Items".  What each function follows:

* ``sort_fixed``      -- Sec. 2.1 (a network's output is the input permutation
  in non-decreasing order) computed by insertion sort "IS Def" (Sec. 4.2), one
  array after another as in the ArrayInRow layout (Sec. 4.1).
* float32 / float64 keys (``sort_fixed``, ``sort_segments``) -- ordered by
  IEEE 754 totalOrder, written case by case from its definition (library
  addition: the paper's keys are integers).
* ``sort_array``     -- one large u32 array, bottom-up merge sort (for the
  large-array sort, where insertion sort would be too slow).
* ``sort_fixed_items`` -- the same for the paper's 16-byte items (u64 key,
  u64 reference, Sec. 4.1), stable by key.
* ``sort_segments``   -- per-segment stable insertion sort; payload values move
  with their keys like the reference values of Sec. 2.2.1.  Ties keep input
  order: the (key, original position) reading of this library.
* ``network_*``       -- comparator semantics, size and depth of Sec. 2.1;
  0-1 inputs (Knuth's 0-1 principle) and all permutations.
* ``perm_product``    -- the probabilistic permutation check of Sec. 4.1.
* ``rss``             -- a step-by-step restatement of Register Sample Sort
  (Sec. 3, Algorithm 1), pure Python, small inputs only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into liboracle.so next to it (idempotent)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = f"{_LIB_PATH}.{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    U64 = ctypes.c_uint64
    I64 = ctypes.c_int64
    for name in ("oracle_sort_fixed_u32", "oracle_sort_fixed_u64"):
        getattr(lib, name).argtypes = [P, I, U64]
        getattr(lib, name).restype = None
    for name in ("oracle_sort_fixed_f32", "oracle_sort_fixed_f64"):
        getattr(lib, name).argtypes = [P, I, U64]
        getattr(lib, name).restype = None
    lib.oracle_sort_array_u32.argtypes = [P, P, U64]
    lib.oracle_sort_array_u32.restype = None
    lib.oracle_sort_fixed_items.argtypes = [P, I, U64]
    lib.oracle_sort_fixed_items.restype = None
    for name in ("oracle_sort_segments_u32", "oracle_sort_segments_u64", "oracle_sort_segments_f32",
                 "oracle_sort_segments_f64"):
        getattr(lib, name).argtypes = [P, P, P, U64]
        getattr(lib, name).restype = None
    for name in ("oracle_network_failures_01", "oracle_network_failures_perm",
                 "oracle_network_failures_01_wide"):
        getattr(lib, name).argtypes = [I, P, P, I]
        getattr(lib, name).restype = I64
    lib.oracle_network_depth.argtypes = [I, P, P, I]
    lib.oracle_network_depth.restype = I
    for name in ("oracle_perm_product_u64", "oracle_perm_product_u32"):
        getattr(lib, name).argtypes = [P, U64, U64, U64]
        getattr(lib, name).restype = U64
    for name in ("oracle_is_sorted_segments_u64", "oracle_is_sorted_segments_u32"):
        getattr(lib, name).argtypes = [P, P, U64]
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def sort_fixed(keys: np.ndarray, n: int) -> np.ndarray:
    """Return a copy of ``keys`` (``count*n`` contiguous u32/u64 keys) with each
    consecutive run of ``n`` keys sorted ascending."""
    lib = _load()
    out = np.ascontiguousarray(keys).copy()
    if out.size % n:
        raise ValueError("size is not a multiple of n")
    fn = {np.dtype(np.uint32): lib.oracle_sort_fixed_u32,
          np.dtype(np.uint64): lib.oracle_sort_fixed_u64,
          np.dtype(np.float32): lib.oracle_sort_fixed_f32,
          np.dtype(np.float64): lib.oracle_sort_fixed_f64}[out.dtype]
    fn(_ptr(out), n, out.size // n)
    return out


def sort_array(keys: np.ndarray) -> np.ndarray:
    """A sorted copy of one u32 array (bottom-up merge sort)."""
    out = np.ascontiguousarray(keys, dtype=np.uint32).copy()
    tmp = np.empty_like(out)
    _load().oracle_sort_array_u32(_ptr(out), _ptr(tmp), out.size)
    return out


def sort_fixed_items(items: np.ndarray, n: int) -> np.ndarray:
    """Return a copy of ``items`` (u64, interleaved key, ref of ``count*n``
    items) with each array of ``n`` items sorted by key, stably (Sec. 4.1)."""
    out = np.ascontiguousarray(items, dtype=np.uint64).copy()
    if out.size % (2 * n):
        raise ValueError("size is not a multiple of 2n")
    _load().oracle_sort_fixed_items(_ptr(out), n, out.size // (2 * n))
    return out


def sort_segments(keys: np.ndarray, vals, offsets: np.ndarray):
    """Stable per-segment sort of CSR segments; returns (keys, vals) copies
    (``vals`` is None when no payload is given)."""
    lib = _load()
    k = np.ascontiguousarray(keys).copy()
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    off = np.ascontiguousarray(offsets, dtype=np.uint32)
    fn = {np.dtype(np.uint32): lib.oracle_sort_segments_u32,
          np.dtype(np.uint64): lib.oracle_sort_segments_u64,
          np.dtype(np.float32): lib.oracle_sort_segments_f32,
          np.dtype(np.float64): lib.oracle_sort_segments_f64}[k.dtype]
    fn(_ptr(k), _ptr(v), _ptr(off), off.size - 1)
    return k, v


def _pairs(pairs):
    lo = np.ascontiguousarray([p[0] for p in pairs], dtype=np.int32)
    hi = np.ascontiguousarray([p[1] for p in pairs], dtype=np.int32)
    return lo, hi


def network_failures_01(n: int, pairs) -> int:
    """Number of 0-1 input vectors the network (0-based (i, j) pairs) fails to sort."""
    lo, hi = _pairs(pairs)
    return int(_load().oracle_network_failures_01(n, _ptr(lo), _ptr(hi), len(lo)))


def network_failures_01_wide(n: int, pairs) -> int:
    """Same count as ``network_failures_01``, 64 vectors per step (7 <= n <= 32)."""
    lo, hi = _pairs(pairs)
    return int(_load().oracle_network_failures_01_wide(n, _ptr(lo), _ptr(hi), len(lo)))


def network_failures_perm(n: int, pairs) -> int:
    """Number of permutations of 0..n-1 the network fails to sort (n <= 10)."""
    lo, hi = _pairs(pairs)
    return int(_load().oracle_network_failures_perm(n, _ptr(lo), _ptr(hi), len(lo)))


def network_depth(n: int, pairs) -> int:
    """Depth of the network (Sec. 2.1)."""
    lo, hi = _pairs(pairs)
    return int(_load().oracle_network_depth(n, _ptr(lo), _ptr(hi), len(lo)))


# Permutation check constants: p is a large prime (Sec. 4.1 leaves the prime
# open); z is arbitrary and is increased until v != 0.
PERM_P = (1 << 61) - 1
PERM_Z = 0x2545F4914F6CDD1D % PERM_P


def perm_product(a: np.ndarray, z: int = PERM_Z, p: int = PERM_P) -> int:
    """v = prod (z - a_i) mod p over all elements of ``a`` (Sec. 4.1)."""
    lib = _load()
    a = np.ascontiguousarray(a)
    fn = {np.dtype(np.uint32): lib.oracle_perm_product_u32,
          np.dtype(np.uint64): lib.oracle_perm_product_u64}[a.dtype]
    return int(fn(_ptr(a), a.size, z, p))


def perm_check_z(a: np.ndarray, p: int = PERM_P) -> int:
    """The z of Sec. 4.1: start at PERM_Z and increment until v != 0."""
    z = PERM_Z
    while perm_product(a, z, p) == 0:
        z += 1
    return z


def is_sorted_segments(keys: np.ndarray, offsets: np.ndarray) -> bool:
    lib = _load()
    k = np.ascontiguousarray(keys)
    off = np.ascontiguousarray(offsets, dtype=np.uint32)
    fn = {np.dtype(np.uint32): lib.oracle_is_sorted_segments_u32,
          np.dtype(np.uint64): lib.oracle_is_sorted_segments_u64}[k.dtype]
    return bool(fn(_ptr(k), _ptr(off), off.size - 1))
