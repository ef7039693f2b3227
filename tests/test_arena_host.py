"""The request server's device-memory allocator (csrc/sn_arena.h, host C++),
compiled with g++ and checked against a brute-force bitmap model of first fit."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


def test_range_arena_matches_first_fit_model(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = os.path.join(tmp_path, "arena_check")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2002_05599_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "native", "arena_check.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "ok"
