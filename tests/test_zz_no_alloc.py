"""pc_inspect_static -- the inspection entry point that allocates no device
memory, for callers that cannot call cudaMalloc (their framework's pool
allocator owns the device, or an allocation could synchronise the device in a
latency-critical loop).  Its scratch is a static device array shared by all
calls.  It must give the same results as pc_inspect, call after call: the
second call checks that the array's leftover contents from the first do not
leak into the next result.

This file is collected last so that a failure here cannot hide the other
tests in a run that stops at the first failure.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import pytest

import oracle
import paper_1401_2130_gb300 as pc

pytestmark = pytest.mark.gpu

MASS_TOL = 1e-5  # the tolerance the parity tests use for the FP32 mass


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    pc.build()
    pc.load()
    torch.cuda.init()


def _call_static(W, L, p, seed, cfg0, n):
    """Call the C entry point directly through ctypes."""
    lib = pc.load()
    v = np.zeros(n, np.uint8); fh = np.zeros(n, np.int32)
    ms = np.zeros(n, np.int32); mass = np.zeros(n, np.float32)
    npc = ctypes.c_int64(-1); pi = ctypes.c_double(-1.0)
    st = lib.pc_inspect_static(W, L, p, seed, cfg0, n, v.ctypes.data, fh.ctypes.data,
                               mass.ctypes.data, ms.ctypes.data, ctypes.addressof(npc),
                               ctypes.addressof(pi), None)
    assert st == pc.PC_OK, lib.pc_last_error()
    return {"verdict": v, "first_hit": fh, "m_stop": ms, "mass": mass,
            "n_percolating": npc.value, "Pi": pi.value}


def _same(a, b):
    for k in ("verdict", "first_hit", "m_stop"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    assert np.abs(np.asarray(a["mass"], np.float64) - np.asarray(b["mass"], np.float64)).max() <= MASS_TOL
    assert a["n_percolating"] == b["n_percolating"]


def test_static_entry_point_matches_pc_inspect_twice():
    # two calls in a row with different lattices and probabilities: the second
    # reuses the static array the first one left behind
    for (W, L, p, seed, cfg0, n) in [(8, 64, 0.2, 2, 0, 3000), (4, 16, 0.3, 1, 500, 2000)]:
        ref = pc.pc_inspect(W, L, p, seed, cfg0, n)
        got = _call_static(W, L, p, seed, cfg0, n)
        _same(got, ref)
        assert got["n_percolating"] > 0


def test_static_entry_point_rejects_oversized_requests():
    lib = pc.load()
    v = np.zeros(4, np.uint8)
    for (W, L, n) in [(8, 64, (1 << 18) + 1), (52, 1, 4), (8, 4096, 4)]:
        st = lib.pc_inspect_static(W, L, 0.2, 1, 0, n, v.ctypes.data, None, None, None,
                                   None, None, None)
        assert st == pc.PC_ERR_ARG
        assert lib.pc_last_error()


@pytest.mark.parametrize("W,L,p,n", [
    (26, 1, 0.5, 400),    # the widest lattice the resident solver holds
    (20, 8, 0.3, 300),    # W = 20: its longest resident fibre
    (12, 33, 0.2, 300),   # W = 12: its longest resident fibre
    (8, 74, 0.21, 400),   # W = 8: its longest resident fibre
])
def test_static_entry_point_matches_the_oracle(W, L, p, n):
    """The static tables are built on the device by their own kernel, so they
    are checked against the CPU oracle directly: verdicts, first hits and
    step counts exact, FP32 mass within 1e-5 absolute and, where the FP64
    mass exceeds 1e-30, within the relative bound of the parity tests
    ((3 + 7 (first_hit - 1) + ceil(P / 32) + 10) 2^-24, times 1.01)."""
    got = _call_static(W, L, p, 17, 0, n)
    ref = oracle.inspect(W, L, p=p, seed=17, n=n, mode="markov", threads=os.cpu_count() or 1)
    assert np.array_equal(got["verdict"].astype(np.int32), ref["verdict"])
    assert np.array_equal(got["first_hit"], ref["first_hit"])
    assert np.array_equal(got["m_stop"], ref["m_stop"])
    mg, mr = got["mass"].astype(np.float64), ref["mass"]
    assert np.abs(mg - mr).max() <= MASS_TOL
    sel = mr > 1e-30
    P = pc.pc_lattice_layout(W)["P"]
    fh = np.maximum(ref["first_hit"][sel], 1)
    tol = 1.01 * (3 + 7 * (fh - 1) + (P + 31) // 32 + 10) * 2.0 ** -24
    assert np.all(np.abs(mg[sel] - mr[sel]) <= tol * mr[sel])
    assert got["n_percolating"] == int(ref["verdict"].sum())
    assert ref["verdict"].sum() > 0
