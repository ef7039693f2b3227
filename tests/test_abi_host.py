"""Host-side checks of the C ABI: the library builds and loads without a GPU,
exports every entry point include/*.h declares, and rejects bad arguments
synchronously, before touching the device."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_2002_05599_gb300 import build as native
    path = native.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("defined",):
                names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sn_sort_fixed", "sn_sort_segments", "rss_sort_segments", "sn_check",
                     "sn_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    lib.sn_status_string.restype = ctypes.c_char_p
    assert lib.sn_status_string(0) == b"ok"
    for code in range(-6, 0):
        assert lib.sn_status_string(code) not in (b"", b"unknown status")


def _call(lib, name, *args):
    fn = getattr(lib, name)
    return fn(*args)


def test_fixed_argument_errors(lib):
    P, U64 = ctypes.c_void_p, ctypes.c_uint64
    for name in ("sn_sort_fixed", "sn_sort_fixed_u64"):
        fn = getattr(lib, name)
        fn.argtypes = [P, ctypes.c_int, U64, P]
        assert fn(None, 1, 10, None) == -1      # n below 2
        assert fn(None, 17, 10, None) == -1     # n above 16
        assert fn(None, 8, 0, None) == 0        # nothing to do, no launch
        assert fn(None, 8, 10, None) == -1      # null keys
        assert fn(0x1000, 16, 1 << 60, None) == -2  # count * n overflows
        assert fn(0x1001, 8, 10, None) == -1    # keys not naturally aligned


def test_segment_argument_errors(lib):
    P, U64 = ctypes.c_void_p, ctypes.c_uint64
    for name in ("sn_sort_segments", "sn_sort_segments_u64", "rss_sort_segments", "rss_sort_segments_u64"):
        fn = getattr(lib, name)
        fn.argtypes = [P, P, P, U64, P]
        assert fn(None, None, None, 0, None) == 0          # empty batch
        assert fn(None, None, 0x1000, 5, None) == -1       # null keys
        assert fn(0x1000, None, None, 5, None) == -1       # null offsets
        assert fn(0x1000, None, 0x2000, 1 << 32, None) == -2  # too many segments
        assert fn(0x1000, 0x3002, 0x2000, 5, None) == -1   # payload misaligned


def test_no_gpu_is_a_clean_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    fn = lib.sn_sort_fixed
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p]
    assert fn(0x1000, 8, 10, None) in (-4, -6)
