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
    for required in ("sn_sort_fixed", "sn_sort_fixed_u64", "sn_sort_segments", "sn_sort_segments_u64",
                     "rss_sort_segments", "rss_sort_segments_u64", "sn_get_last_cuda_error", "sn_tune", "sn_check",
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


def test_server_argument_errors(lib):
    from paper_2002_05599_gb300.server import ServerConfig
    P = ctypes.c_void_p
    create = lib.sn_server_create
    create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(P)]
    h = P()
    assert create(None, ctypes.byref(h)) == -1
    for bad in (ServerConfig(1 << 20, 2, 4, 0, 0, 0),       # key_bytes not 4 or 8
                ServerConfig(1 << 20, 4, 17, 0, 0, 0),      # too many slots
                ServerConfig(1 << 20, 4, 4, 1 << 40, 0, 0),  # batch key limit above 2^31
                ServerConfig(1 << 20, 4, 4, 0, 0, 100000),  # too many requests per batch
                ServerConfig(16, 4, 4, 0, 0, 0)):           # budget below one allocation unit
        assert create(ctypes.byref(bad), ctypes.byref(h)) == -1
        assert not h.value
    submit = lib.sn_server_submit
    submit.argtypes = [P, P, P, P, ctypes.c_uint64, P, P, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]
    t = ctypes.c_uint64()
    assert submit(None, None, None, None, 0, None, None, 0, ctypes.byref(t)) == -1
    for name in ("sn_server_drain", "sn_server_destroy"):
        getattr(lib, name).argtypes = [P]
        assert getattr(lib, name)(None) == -1
    lib.sn_server_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_int64]
    assert lib.sn_server_wait(None, 1, 0) == -1
    import torch
    if not torch.cuda.is_available():  # a valid config still needs the GPU
        assert create(ctypes.byref(ServerConfig(1 << 20, 4, 4, 0, 0, 0)), ctypes.byref(h)) in (-4, -6)


def test_tile_shape_limits(lib):
    # Shared-memory and task-ring limits of the tile shapes, checked before any
    # device is touched (a shape that passes gets past SN_EINVAL; on a machine
    # without a GPU the call then fails on the device instead).  Ring kernel:
    # a packed stage takes max(6, key + payload bytes) per unit of
    # tile_units + 256 bytes; synchronous kernel: fixed regions.
    import paper_2002_05599_gb300 as sn
    from paper_2002_05599_gb300._binding import SnTuning
    L = sn._binding._tune_lib()

    def fits(kb, vals, units, stages, mode=0):
        return L.sn_tuning_set(kb, vals, ctypes.byref(SnTuning(units, 0x1F, 160, stages, mode))) != -1

    assert fits(4, 0, 16384, 2) and not fits(4, 0, 16384, 3)    # 6 B per unit
    assert fits(4, 0, 8192, 4)
    for kb, v in ((4, 1), (8, 0)):                               # 8 B per unit
        assert fits(kb, v, 8192, 3) and not fits(kb, v, 8192, 4)
        assert not fits(kb, v, 16384, 2)
    assert fits(8, 1, 8192, 2) and not fits(8, 1, 8192, 3)      # 12 B per unit
    assert fits(8, 1, 6144, 2) and fits(8, 1, 4096, 4)
    assert fits(4, 0, 8192, 2, 1)                                # synchronous kernel
    for kb, v in ((4, 1), (8, 0), (8, 1)):
        assert not fits(kb, v, 8192, 2, 1) and fits(kb, v, 4096, 2, 1)
    assert not fits(4, 0, 32768, 2) and not fits(4, 0, 256, 2)
    # window kernel (mode 2): four warps a block, each with `stages` windows of
    # tile_units items (key + payload bytes each) plus its sample-sort scratch
    assert fits(4, 0, 4096, 3, 2) and not fits(4, 0, 4096, 4, 2)   # 4 B per item
    assert fits(8, 1, 2048, 2, 2) and not fits(8, 1, 2048, 3, 2)   # 12 B per item
    assert fits(8, 1, 1024, 4, 2) and not fits(8, 1, 8192, 2, 2) and not fits(4, 0, 256, 2, 2)
    for kb in (4, 8):  # on a GPU machine the shapes above were installed: back to the defaults
        for v in (False, True):
            sn.sn_tuning_set(kb, v)


def test_tuning_argument_errors_and_file_format(lib, tmp_path):
    import paper_2002_05599_gb300 as sn
    from paper_2002_05599_gb300._binding import SnTuning
    L = sn._binding._tune_lib()
    t = SnTuning(2048, 0xF, 160, 2, 0)
    assert L.sn_tuning_set(2, 0, ctypes.byref(t)) == -1            # key_bytes
    assert L.sn_tuning_get(4, 0, None) == -1
    for bad in (SnTuning(256, 0xF, 160, 2, 0), SnTuning(32768, 0xF, 160, 2, 0), SnTuning(2048, 0x20, 160, 2, 0),
                SnTuning(2048, 0xF, 8, 2, 0), SnTuning(2048, 0xF, 300, 2, 0), SnTuning(2048, 0xF, 160, 1, 0),
                SnTuning(2048, 0xF, 160, 5, 0), SnTuning(2048, 0xF, 160, 2, 3),
                SnTuning(8192, 0xF, 160, 4, 0), SnTuning(8192, 0xF, 160, 2, 1),   # staging too large
                SnTuning(8192, 0xF, 160, 2, 2), SnTuning(4096, 0xF, 160, 4, 2)):  # window too large
        assert L.sn_tuning_set(4, 1, ctypes.byref(bad)) == -1
    L.sn_tune_segments.argtypes = L.sn_tune_segments.argtypes
    assert L.sn_tune_segments(None, None, None, 5, 4, None, None, None) == -1
    assert L.sn_tune_segments(0x1000, None, 0x2000, 5, 3, None, None, None) == -1
    assert L.sn_tune_rss_segments(None, None, None, 5, 4, None, None, None) == -1
    assert L.sn_tune_rss_segments(0x1000, None, 0x2000, 5, 3, None, None, None) == -1
    assert sn.sn_tuning_save(os.path.join(tmp_path, "no", "such", "dir.txt")) == -1
    bad_file = os.path.join(tmp_path, "bad.txt")
    with open(bad_file, "w") as f:
        f.write("smallsort-tuning 3\n0 4 0 2048 15 160 2\n")  # truncated line
    assert sn.sn_tuning_load(bad_file) == -1
    with open(bad_file, "w") as f:
        f.write("smallsort-tuning 3\n0 4 0 100 15 160 2 0\n")  # tile size out of range
    assert sn.sn_tuning_load(bad_file) == -1
    with open(bad_file, "w") as f:
        f.write("smallsort-tuning 3\n0 8 1 8192 15 160 3 0\n")  # three 8192-unit stages do not fit
    assert sn.sn_tuning_load(bad_file) == -1
    with open(bad_file, "w") as f:
        f.write("smallsort-tuning 2\n0 4 0 2048 15 160 2\n")  # old format
    assert sn.sn_tuning_load(bad_file) == -1
    assert sn.sn_tuning_load(os.path.join(tmp_path, "missing.txt")) == -1
    good = os.path.join(tmp_path, "good.txt")
    with open(good, "w") as f:
        f.write("smallsort-tuning 3\n0 4 0 4096 5 128 2 1\n0 8 1 1024 15 192 4 0\n")
    assert sn.sn_tuning_load(good) == 0  # entries for devices that are not present are skipped
