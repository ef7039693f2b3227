"""ctypes binding of the request server (include/smallsort_server.h).

Marshalling only: the queue, admission by device-memory budget, coalescing,
the copies and the sorts all run in libsmallsort.so.  Request buffers are
host arrays (numpy arrays or CPU tensors; pinned memory makes the copies
asynchronous); the binding keeps a reference to them until the request has
been collected with ``wait`` so they cannot be freed while the GPU uses them.
"""
from __future__ import annotations

import ctypes
import threading

from ._binding import SN_OK, SmallSortError, library

_U64, _I, _U32, _D = ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, ctypes.c_double


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", _U64), ("key_bytes", _I), ("slots", _I), ("max_batch_keys", _U64),
                ("max_batch_segments", _U64), ("max_batch_requests", _U32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", _U64), ("completed", _U64), ("failed", _U64), ("batches", _U64),
                ("keys_completed", _U64), ("segments_completed", _U64), ("max_batch_requests_seen", _U64),
                ("max_inflight_seen", _U32), ("pad", _U32), ("peak_device_bytes", _U64),
                ("latency_p50_us", _D), ("latency_p99_us", _D), ("latency_max_us", _D),
                ("latency_mean_us", _D), ("span_s", _D), ("keys_per_s", _D)]


_bound = False


def _lib():
    global _bound
    lib = library()
    if not _bound:
        P = ctypes.c_void_p
        lib.sn_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(P)]
        lib.sn_server_submit.argtypes = [P, P, P, P, _U64, P, P, ctypes.c_int64, ctypes.POINTER(_U64)]
        lib.sn_server_wait.argtypes = [P, _U64, ctypes.c_int64]
        lib.sn_server_drain.argtypes = [P]
        lib.sn_server_stats_get.argtypes = [P, ctypes.POINTER(ServerStats), _I]
        lib.sn_server_destroy.argtypes = [P]
        lib.sn_server_now_ns.argtypes = []
        lib.sn_server_now_ns.restype = ctypes.c_int64
        for name in ("sn_server_create", "sn_server_submit", "sn_server_wait", "sn_server_drain",
                     "sn_server_stats_get", "sn_server_destroy"):
            getattr(lib, name).restype = _I
        _bound = True
    return lib


def now_ns() -> int:
    """The server's monotonic clock (arrival times for ``submit``)."""
    return int(_lib().sn_server_now_ns())


def _host_addr(a, size: int | None = None):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor
        if a.is_cuda:
            raise ValueError("server requests take host buffers")
        if not a.is_contiguous():
            raise ValueError("expected a contiguous buffer")
        if size is not None and a.element_size() != size:
            raise ValueError(f"expected {size}-byte elements")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a contiguous buffer")
    if size is not None and a.itemsize != size:
        raise ValueError(f"expected {size}-byte elements")
    return a.ctypes.data


class SortServer:
    """Continuous-batching sort server on the current CUDA device."""

    def __init__(self, budget_bytes: int, key_bytes: int = 4, slots: int = 4, max_batch_keys: int = 0,
                 max_batch_segments: int = 0, max_batch_requests: int = 0):
        self.key_bytes = key_bytes
        cfg = ServerConfig(budget_bytes, key_bytes, slots, max_batch_keys, max_batch_segments, max_batch_requests)
        h = ctypes.c_void_p()
        rc = _lib().sn_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != SN_OK:
            raise SmallSortError(rc, "sn_server_create")
        self._h = h
        self._keep = {}
        self._mu = threading.Lock()

    def submit(self, keys_in, offsets, vals_in=None, keys_out=None, vals_out=None, arrival_ns: int = 0) -> int:
        """Queue one request; returns its ticket (raises on a rejected request)."""
        if keys_out is None:
            keys_out = keys_in
        if vals_in is not None and vals_out is None:
            vals_out = vals_in
        nseg = (offsets.numel() if hasattr(offsets, "numel") else offsets.size) - 1
        t = _U64()
        rc = _lib().sn_server_submit(self._h, _host_addr(keys_in, self.key_bytes), _host_addr(vals_in, 4),
                                     _host_addr(offsets, 4), max(nseg, 0), _host_addr(keys_out, self.key_bytes),
                                     _host_addr(vals_out, 4), arrival_ns, ctypes.byref(t))
        if rc != SN_OK:
            raise SmallSortError(rc, "sn_server_submit")
        with self._mu:
            self._keep[t.value] = (keys_in, offsets, vals_in, keys_out, vals_out)
        return t.value

    def wait(self, ticket: int, timeout_ns: int = -1) -> int:
        """Status of a finished request (SN_ETIMEOUT while it runs)."""
        rc = _lib().sn_server_wait(self._h, ticket, timeout_ns)
        if rc != -5:  # anything but "still running" collects the ticket
            with self._mu:
                self._keep.pop(ticket, None)
        return rc

    def drain(self) -> None:
        _lib().sn_server_drain(self._h)

    def stats(self, reset: bool = False) -> dict:
        st = ServerStats()
        _lib().sn_server_stats_get(self._h, ctypes.byref(st), 1 if reset else 0)
        return {name: getattr(st, name) for name, _ in ServerStats._fields_ if name != "pad"}

    def close(self) -> None:
        if self._h:
            _lib().sn_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
