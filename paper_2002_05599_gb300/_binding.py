"""ctypes binding of libsmallsort.so (same names as include/smallsort.h).

Marshalling only: tensors become device addresses and element counts, the
stream defaults to torch's current CUDA stream.  There is no CPU fallback: if
the library is missing the first call raises.
"""
from __future__ import annotations

import ctypes
import os

SN_OK = 0
SN_EINVAL = -1
SN_ERANGE = -2
SN_ENOMEM = -3
SN_ECUDA = -4
SN_ETIMEOUT = -5
SN_EUNSUPPORTED = -6

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsmallsort.so")
_lib = None


class SmallSortError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {sn_status_string(status)} ({status})" if what else
                         f"{sn_status_string(status)} ({status})")


def library_path() -> str:
    return _LIB_PATH


def library():
    """Load libsmallsort.so (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(_LIB_PATH)
    P, U64, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    lib.sn_sort_fixed.argtypes = [P, I, U64, P]
    lib.sn_sort_fixed_u64.argtypes = [P, I, U64, P]
    lib.sn_sort_fixed_family.argtypes = [P, I, U64, I, P]
    lib.sn_sort_fixed_items.argtypes = [P, I, U64, I, P]
    lib.sn_sort_fixed_family.restype = I
    lib.sn_sort_fixed_items.restype = I
    for name in ("sn_sort_fixed_f32", "sn_sort_fixed_f64"):
        getattr(lib, name).argtypes = [P, I, U64, P]
        getattr(lib, name).restype = I
    for name in ("sn_sort_segments_f32", "sn_sort_segments_f64", "sn_sort_segments_large",
                 "sn_sort_segments_large_u64"):
        getattr(lib, name).argtypes = [P, P, P, U64, P]
        getattr(lib, name).restype = I
    for name in ("sn_sort_segments", "sn_sort_segments_u64",
                 "rss_sort_segments", "rss_sort_segments_u64"):
        getattr(lib, name).argtypes = [P, P, P, U64, P]
    lib.sn_check.argtypes = [P]
    lib.sn_status_string.argtypes = [I]
    lib.sn_status_string.restype = ctypes.c_char_p
    for name in ("sn_sort_fixed", "sn_sort_fixed_u64", "sn_sort_segments", "sn_sort_segments_u64",
                 "rss_sort_segments", "rss_sort_segments_u64", "sn_check"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def _addr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _elems(x, size: int) -> int:
    if x.element_size() != size:
        raise ValueError(f"expected {size}-byte elements, got {x.element_size()}")
    return x.numel()


def sn_sort_fixed(keys, n: int, count: int | None = None, stream=None) -> int:
    """Sort ``count`` contiguous arrays of ``n`` u32 keys in place."""
    if count is None:
        count = _elems(keys, 4) // n
    return library().sn_sort_fixed(_addr(keys), n, count, _stream(stream))


def sn_sort_fixed_u64(keys, n: int, count: int | None = None, stream=None) -> int:
    """Sort ``count`` contiguous arrays of ``n`` u64 keys in place."""
    if count is None:
        count = _elems(keys, 8) // n
    return library().sn_sort_fixed_u64(_addr(keys), n, count, _stream(stream))


SN_NETWORK_BEST = 0
SN_NETWORK_BOSE_NELSON = 1


def sn_sort_fixed_family(keys, n: int, family: int, count: int | None = None, stream=None) -> int:
    """sn_sort_fixed with a network family (SN_NETWORK_BEST / SN_NETWORK_BOSE_NELSON)."""
    if count is None:
        count = _elems(keys, 4) // n
    return library().sn_sort_fixed_family(_addr(keys), n, count, family, _stream(stream))


def sn_sort_fixed_items(items, n: int, family: int = SN_NETWORK_BEST, count: int | None = None,
                        stream=None) -> int:
    """Sort ``count`` arrays of ``n`` 16-byte items (u64 key, u64 ref; a 64-bit
    tensor of 2*count*n elements, key and ref interleaved) by key, in place."""
    if count is None:
        count = _elems(items, 8) // (2 * n)
    return library().sn_sort_fixed_items(_addr(items), n, count, family, _stream(stream))


def sn_sort_fixed_f32(keys, n: int, count: int | None = None, stream=None) -> int:
    """Sort ``count`` arrays of ``n`` float32 keys in place (IEEE 754 totalOrder)."""
    if count is None:
        count = _elems(keys, 4) // n
    return library().sn_sort_fixed_f32(_addr(keys), n, count, _stream(stream))


def sn_sort_fixed_f64(keys, n: int, count: int | None = None, stream=None) -> int:
    """Sort ``count`` arrays of ``n`` float64 keys in place (IEEE 754 totalOrder)."""
    if count is None:
        count = _elems(keys, 8) // n
    return library().sn_sort_fixed_f64(_addr(keys), n, count, _stream(stream))


def sn_sort_segments_f32(keys, vals, offsets, nseg: int | None = None, stream=None) -> int:
    return _segments(library().sn_sort_segments_f32, 4, keys, vals, offsets, nseg, stream)


def sn_sort_segments_f64(keys, vals, offsets, nseg: int | None = None, stream=None) -> int:
    return _segments(library().sn_sort_segments_f64, 8, keys, vals, offsets, nseg, stream)


SN_MAX_SEGMENT_LARGE = 4096


def sn_sort_large(keys, n: int | None = None, stream=None) -> int:
    """Sort one array of u32 keys (sample-sort partition + segmented base case); synchronous."""
    lib = library()
    if not getattr(lib, "_large_bound", False):
        lib.sn_sort_large.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
        lib.sn_sort_large.restype = ctypes.c_int
        lib._large_bound = True
    if n is None:
        n = _elems(keys, 4)
    return lib.sn_sort_large(_addr(keys), n, _stream(stream))


def sn_sort_segments_large(keys, vals, offsets, nseg: int | None = None, stream=None) -> int:
    """Segments of up to SN_MAX_SEGMENT_LARGE u32 keys (one thread block per segment)."""
    return _segments(library().sn_sort_segments_large, 4, keys, vals, offsets, nseg, stream)


def sn_sort_segments_large_u64(keys, vals, offsets, nseg: int | None = None, stream=None) -> int:
    return _segments(library().sn_sort_segments_large_u64, 8, keys, vals, offsets, nseg, stream)


def _segments(fn, ksize, keys, vals, offsets, nseg, stream):
    if nseg is None:
        nseg = _elems(offsets, 4) - 1
    if not isinstance(keys, int):
        _elems(keys, ksize)
    if vals is not None and not isinstance(vals, int):
        _elems(vals, 4)
    return fn(_addr(keys), _addr(vals), _addr(offsets), nseg, _stream(stream))


def sn_sort_segments(keys, vals, offsets, nseg: int | None = None, stream=None) -> int:
    return _segments(library().sn_sort_segments, 4, keys, vals, offsets, nseg, stream)


def sn_sort_segments_u64(keys, vals, offsets, nseg: int | None = None, stream=None) -> int:
    return _segments(library().sn_sort_segments_u64, 8, keys, vals, offsets, nseg, stream)


def rss_sort_segments(keys, vals, offsets, nseg: int | None = None, stream=None) -> int:
    return _segments(library().rss_sort_segments, 4, keys, vals, offsets, nseg, stream)


def rss_sort_segments_u64(keys, vals, offsets, nseg: int | None = None, stream=None) -> int:
    return _segments(library().rss_sort_segments_u64, 8, keys, vals, offsets, nseg, stream)


class SnTuning(ctypes.Structure):
    _fields_ = [("tile_units", ctypes.c_int), ("net_classes", ctypes.c_uint), ("rss_two_min", ctypes.c_int),
                ("tile_stages", ctypes.c_int), ("tile_mode", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {"tile_units": self.tile_units, "net_classes": self.net_classes, "rss_two_min": self.rss_two_min,
                "tile_stages": self.tile_stages, "tile_mode": self.tile_mode}


def _tune_lib():
    lib = library()
    if not getattr(lib, "_tune_bound", False):
        P = ctypes.c_void_p
        lib.sn_tuning_get.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(SnTuning)]
        lib.sn_tuning_set.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(SnTuning)]
        for name in ("sn_tune_segments", "sn_tune_rss_segments"):
            getattr(lib, name).argtypes = [P, P, P, ctypes.c_uint64, ctypes.c_int, P, ctypes.POINTER(SnTuning),
                                           ctypes.POINTER(ctypes.c_float)]
        lib.sn_tuning_save.argtypes = [ctypes.c_char_p]
        lib.sn_tuning_load.argtypes = [ctypes.c_char_p]
        for name in ("sn_tuning_get", "sn_tuning_set", "sn_tune_segments", "sn_tune_rss_segments", "sn_tuning_save",
                     "sn_tuning_load"):
            getattr(lib, name).restype = ctypes.c_int
        lib._tune_bound = True
    return lib


def sn_tuning_get(key_bytes: int, with_vals: bool) -> dict:
    t = SnTuning()
    check(_tune_lib().sn_tuning_get(key_bytes, int(with_vals), ctypes.byref(t)), "sn_tuning_get")
    return t.as_dict()


def sn_tuning_set(key_bytes: int, with_vals: bool, tile_units: int = 4096, net_classes: int = 0x1F,
                  rss_two_min: int = 160, tile_stages: int = 2, tile_mode: int = 0) -> int:
    t = SnTuning(tile_units, net_classes, rss_two_min, tile_stages, tile_mode)
    return _tune_lib().sn_tuning_set(key_bytes, int(with_vals), ctypes.byref(t))


def sn_tune_segments(keys, vals, offsets, nseg: int | None = None, stream=None, rss_only: bool = False):
    """Autotune the segmented call (rss_sort_segments* if rss_only) on this
    batch; returns (parameters, ms of one sort)."""
    if nseg is None:
        nseg = _elems(offsets, 4) - 1
    kb = keys.element_size()
    t, ms = SnTuning(), ctypes.c_float()
    name = "sn_tune_rss_segments" if rss_only else "sn_tune_segments"
    check(getattr(_tune_lib(), name)(_addr(keys), _addr(vals), _addr(offsets), nseg, kb, _stream(stream),
                                     ctypes.byref(t), ctypes.byref(ms)), name)
    return t.as_dict(), float(ms.value)


def sn_tuning_save(path: str) -> int:
    return _tune_lib().sn_tuning_save(os.fsencode(path))


def sn_tuning_load(path: str) -> int:
    return _tune_lib().sn_tuning_load(os.fsencode(path))


def sn_tune(path: str | None = None) -> int:
    """Load a saved parameter table from ``path``, or tune every key type and
    payload kind on the library's synthetic batch (and save to ``path``)."""
    lib = _tune_lib()
    lib.sn_tune.argtypes = [ctypes.c_char_p]
    lib.sn_tune.restype = ctypes.c_int
    return lib.sn_tune(None if path is None else os.fsencode(path))


def sn_check(stream=None) -> int:
    """Synchronise the stream; return and clear the device status word."""
    return library().sn_check(_stream(stream))


def sn_get_last_cuda_error() -> int:
    """Synchronise the device; return and clear the device status word."""
    lib = library()
    lib.sn_get_last_cuda_error.argtypes = []
    lib.sn_get_last_cuda_error.restype = ctypes.c_int
    return lib.sn_get_last_cuda_error()


def sn_status_string(status: int) -> str:
    try:
        return library().sn_status_string(status).decode()
    except RuntimeError:
        return {0: "ok", -1: "invalid argument", -2: "size or offsets out of range",
                -3: "device scratch allocation failed", -4: "CUDA error",
                -5: "bounded device wait timed out", -6: "device not supported"}.get(status, "unknown")


def check(status: int, what: str = "") -> None:
    """Raise SmallSortError unless status is SN_OK."""
    if status != SN_OK:
        raise SmallSortError(status, what)
