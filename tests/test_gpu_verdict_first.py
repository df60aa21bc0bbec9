"""PC_VERDICT_FIRST: the reached set decides every configuration first, and
the FP32 recursion then runs only on the configurations that percolate
(their mass is the only non-zero one, Sec. II.B).  The outputs must equal
the single-pass inspection's to the bit, and the oracle's."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
import paper_1401_2130_gb300 as pc

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1
KEYS = ("verdict", "first_hit", "m_stop", "mass")


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    pc.build()
    pc.load()
    torch.cuda.init()


def _identical(a, b, what):
    for k in KEYS:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), f"{what}: {k}"
    assert a["n_percolating"] == b["n_percolating"], what


@pytest.mark.parametrize("W,L,p,n", [
    (8, 64, 0.17, 2000), (8, 64, 0.19, 2000), (8, 64, 0.2, 4000), (8, 64, 0.3, 500),
    (4, 16, 0.15, 1000), (4, 200, 0.35, 300), (12, 33, 0.2, 300), (3, 2, 0.5, 400),
    (0, 5, 0.9, 300), (5, 3, 0.0, 50), (5, 3, 1.0, 10), (3, 1, 0.4, 100),
])
def test_same_outputs_as_single_pass(W, L, p, n):
    full = pc.pc_inspect(W, L, p, 5, 0, n, mode=pc.PC_MODE_RESIDENT)
    vf = pc.pc_inspect(W, L, p, 5, 0, n, mode=pc.PC_MODE_RESIDENT, verdict_first=True)
    _identical(vf, full, f"W={W} L={L} p={p}")


def test_against_the_oracle():
    """Tiny workload (W = 4, L = 16, p = 0.15, seed 1) and the p-sweep
    lattice at p = 0.2: exact verdicts, first hits and step counts, masses
    within 1e-5 absolute and 1e-4 relative (above 1e-30)."""
    for (W, L, p, seed, n) in [(4, 16, 0.15, 1, 1000), (8, 64, 0.2, 2, 2000)]:
        g = pc.pc_inspect(W, L, p, seed, 0, n, verdict_first=True)
        r = oracle.inspect(W, L, p=p, seed=seed, n=n, mode="markov", threads=THREADS)
        assert np.array_equal(g["verdict"].astype(np.int32), r["verdict"])
        assert np.array_equal(g["first_hit"], r["first_hit"])
        assert np.array_equal(g["m_stop"], r["m_stop"])
        mg = g["mass"].astype(np.float64)
        assert np.abs(mg - r["mass"]).max() <= 1e-5
        sel = r["mass"] > 1e-30
        assert np.all(np.abs(mg[sel] - r["mass"][sel]) <= 1e-4 * r["mass"][sel])


def test_wires_exact():
    """Induced wires on the largest resident lattice of W = 8: the mass at the
    first hit is 2^-(sites-1) exactly."""
    import sys
    import torch
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import _wires
    occ, sites = _wires.wire_occupancies(8, 74, 8, 53)
    bits = torch.from_numpy(oracle.pack_bits(occ).view(np.int32)).cuda()
    g = pc.pc_inspect_occupancy(8, 74, bits, mode=pc.PC_MODE_RESIDENT)
    vf = pc.load().pc_inspect_occupancy  # through the flag on the occupancy entry point
    out = pc._alloc_outputs(len(sites), False, pc.ALL_OUTPUTS)
    import ctypes
    npc = ctypes.c_int64(0)
    st = vf(8, 74, pc._ptr(bits), len(sites), pc._ptr(out["verdict"]), pc._ptr(out["first_hit"]),
            pc._ptr(out["mass"]), pc._ptr(out["m_stop"]), ctypes.addressof(npc), None,
            pc.PC_MODE_RESIDENT | pc.PC_VERDICT_FIRST, None)
    assert st == pc.PC_OK
    assert np.array_equal(out["first_hit"], sites)
    assert np.array_equal(out["mass"].astype(np.float64), 2.0 ** -(sites - 1.0))
    assert np.array_equal(out["mass"], g["mass"])


@pytest.mark.parametrize("W,L,p,n", [
    (8, 90, 0.2, 60),     # verdict pass on a one-CTA cluster
    (20, 300, 0.2, 100),  # two CTAs
    (32, 200, 0.17, 40),  # four CTAs
    (64, 120, 0.16, 12),  # sixteen CTAs
    (65, 40, 0.2, 6),     # wider than a cluster holds: step-synchronous verdict pass
    (20, 64, 0.0, 8),     # nothing percolates: no FP32 pass at all
])
def test_streamed_verdict_first_equals_the_single_pass(W, L, p, n):
    """Streamed path: a verdict-only solve of every configuration, then the
    full solve of the percolating ones (outputs at their own indices)."""
    a = pc.pc_inspect(W, L, p, 7, 3, n, mode=pc.PC_MODE_STREAM)
    b = pc.pc_inspect(W, L, p, 7, 3, n, mode=pc.PC_MODE_STREAM, verdict_first=True)
    _identical(a, b, (W, L, p))


def test_streamed_verdict_first_device_outputs():
    import torch
    W, L, p, n = 20, 150, 0.19, 80
    a = pc.pc_inspect(W, L, p, 9, 0, n, mode=pc.PC_MODE_STREAM)
    b = pc.pc_inspect(W, L, p, 9, 0, n, mode=pc.PC_MODE_STREAM, verdict_first=True, device=True)
    torch.cuda.synchronize()
    b = {k: v.cpu().numpy() for k, v in b.items()}
    for k in KEYS:
        assert np.array_equal(np.asarray(a[k]), b[k]), k
    assert int(b["n_percolating"][0]) == a["n_percolating"]


def test_batch_with_the_flag():
    specs = [(8, 64, 0.2, 2, 0, 1500), (4, 32, 0.2, 2, 0, 1500), (16, 40, 0.17, 3, 0, 40)]
    plain = [pc.pc_inspect(*sp) for sp in specs]
    got, _ = pc.pc_batch_run(specs, verdict_first=True)
    for g, r, sp in zip(got, plain, specs):
        for k in KEYS:
            assert np.array_equal(np.asarray(g[k]), np.asarray(r[k])), (sp, k)
