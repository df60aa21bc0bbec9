"""Host-side parts of the library, compiled with the host C++ compiler (no
GPU): the server's HBM admission allocator (csrc/arena.h) against a granule
model, the autotuner's file format (csrc/tune_file.h), the streamed
solver's tick planner (csrc/plan.h) simulated over many fibre lengths, and
the verdict-only blocked solver's pass planner and mask decoding
(csrc/blocked_plan.h) simulated over fibre lengths, slab heights and
configuration histories."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _compile(tmp_path_factory, name):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp(name) / name)
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-I",
                    os.path.join(ROOT, "paper_1401_2130_gb300", "csrc"),
                    os.path.join(ROOT, "tests", name + ".cpp"), "-o", exe], check=True)
    return exe


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    return _compile(tmp_path_factory, "arena_check")


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_arena_first_fit_and_merging(checker, seed):
    r = subprocess.run([checker, str(seed)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_tune_file_round_trip_and_damaged_entries(tmp_path_factory, tmp_path):
    exe = _compile(tmp_path_factory, "tune_file_check")
    r = subprocess.run([exe, str(tmp_path / "tune.json")], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_tick_planner_keeps_every_read_ready(tmp_path_factory):
    exe = _compile(tmp_path_factory, "plan_check")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout[-3000:] + r.stderr


def test_blocked_pass_planner_and_outcomes(tmp_path_factory):
    exe = _compile(tmp_path_factory, "blocked_plan_check")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout[-3000:] + r.stderr
