"""The server's HBM admission allocator (csrc/arena.h, host code) against a
granule model, compiled with the host C++ compiler: no GPU needed."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("arena") / "arena_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-I",
                    os.path.join(ROOT, "paper_1401_2130_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "arena_check.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_arena_first_fit_and_merging(checker, seed):
    r = subprocess.run([checker, str(seed)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
