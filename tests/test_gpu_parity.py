"""GPU parity: libpercol (through its C ABI) against the CPU oracle.

Verdicts, first_hit and m_stop are compared bit-exact on every configuration;
the FP32 detector mass against the oracle's FP64 within the absolute
tolerance 1e-5.  Occupancy bits are compared bit-exact.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
import paper_1401_2130_gb300 as pc

pytestmark = pytest.mark.gpu

MASS_TOL = 1e-5  # absolute, FP32 path vs FP64 oracle
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    pc.build()
    pc.load()
    torch.cuda.init()
    yield
    torch.cuda.synchronize()


def _host(o):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in o.items()}


def assert_parity(gpu, ref, mass=True, what=""):
    v = np.asarray(gpu["verdict"]).astype(np.int32)
    assert np.array_equal(v, ref["verdict"]), f"{what}: verdicts differ at {np.flatnonzero(v != ref['verdict'])[:10]}"
    assert np.array_equal(np.asarray(gpu["first_hit"]), ref["first_hit"]), what
    assert np.array_equal(np.asarray(gpu["m_stop"]), ref["m_stop"]), what
    if mass:
        err = np.abs(np.asarray(gpu["mass"]).astype(np.float64) - ref["mass"])
        assert err.max(initial=0.0) <= MASS_TOL, f"{what}: mass error {err.max()}"


# ---------------------------------------------------------------------------
# occupancy stream
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("W,L,p,seed,cfg0,n", [
    (4, 16, 0.15, 1, 0, 64),        # tiny
    (8, 64, 0.2, 2, 1000, 16),      # p-sweep lattice
    (3, 7, 0.5, 9, 3, 33),          # N = 259: ragged last word
    (0, 1, 1.0, 5, 0, 4),           # one site, every site metallic
    (2, 3, 0.0, 5, 0, 4),           # p = 0
    (64, 40, 0.1533, 4, 7, 2),      # wide lattice
])
def test_occupancy_bits_bit_exact(W, L, p, seed, cfg0, n):
    import torch
    bits = pc.pc_occupancy(W, L, p, seed, cfg0, n)
    torch.cuda.synchronize()
    got = bits.cpu().numpy().view(np.uint32)
    ref = oracle.pack_bits(oracle.occupancy(W, L, p, seed, cfg0, n))
    assert np.array_equal(got, ref)


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

def test_tiny_workload_every_config():
    """W = 4, L = 16, p = 0.15, 1000 configurations, seed 1."""
    W, L, p, seed, n = 4, 16, 0.15, 1, 1000
    g = pc.pc_inspect(W, L, p, seed, 0, n)
    ref = oracle.inspect(W, L, p=p, seed=seed, n=n, mode="markov", threads=THREADS)
    bfs = oracle.inspect(W, L, p=p, seed=seed, n=n, mode="bfs", threads=THREADS)
    assert_parity(g, ref, what="tiny")
    assert np.array_equal(ref["verdict"], bfs["verdict"])
    assert g["n_percolating"] == int(ref["verdict"].sum())
    assert g["Pi"] == ref["verdict"].sum() / n


def test_psweep_workload_every_config():
    """W = 8, L = 64, p = 0.100 .. 0.200 step 0.005, 10^4 configurations per p,
    seed 2, one launch per p with device outputs (the benchmark's launch
    configuration); every configuration against the FP64 Markov oracle."""
    import torch
    W, L, seed, n = 8, 64, 2, 10_000
    for k in range(21):
        p = round(0.100 + 0.005 * k, 3)
        g = pc.pc_inspect(W, L, p, seed, 0, n, device=True)
        torch.cuda.synchronize()
        g = _host(g)
        ref = oracle.inspect(W, L, p=p, seed=seed, n=n, mode="markov", threads=THREADS)
        assert_parity(g, ref, what=f"p={p}")
        assert int(g["n_percolating"][0]) == int(ref["verdict"].sum())


def _all_patterns(N):
    k = np.arange(2**N, dtype=np.uint32)
    return ((k[:, None] >> np.arange(N, dtype=np.uint32)) & 1).astype(np.uint8)


@pytest.mark.parametrize("mode", [0, pc.PC_MODE_STREAM])
def test_every_configuration_of_a_tiny_lattice(mode):
    """All 2^14 occupancies of W = 1, L = 2 through pc_inspect_occupancy."""
    import torch
    W, L = 1, 2
    occ = _all_patterns(14)
    bits = torch.from_numpy(oracle.pack_bits(occ).view(np.int32)).cuda()
    g = pc.pc_inspect_occupancy(W, L, bits, mode=mode)
    ref = oracle.inspect(W, L, occ=occ, mode="markov", threads=THREADS)
    assert_parity(g, ref, what="brute force")


def test_random_explicit_occupancies_ragged():
    import torch
    rng = np.random.default_rng(3)
    for W, L in [(2, 9), (5, 11), (7, 33)]:
        A, N = oracle.lattice_info(W, L)
        occ = (rng.random((200, N)) < 0.45).astype(np.uint8)
        bits = torch.from_numpy(oracle.pack_bits(occ).view(np.int32)).cuda()
        g = pc.pc_inspect_occupancy(W, L, bits)
        ref = oracle.inspect(W, L, occ=occ, mode="markov", threads=THREADS)
        assert_parity(g, ref, what=f"explicit W={W} L={L}")


# ---------------------------------------------------------------------------
# streamed solver
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("W,L,p,n", [(4, 16, 0.3, 300), (8, 64, 0.19, 400), (3, 40, 0.45, 200)])
def test_stream_mode_matches_resident_and_oracle(W, L, p, n):
    res = pc.pc_inspect(W, L, p, 11, 0, n, mode=pc.PC_MODE_RESIDENT)
    stm = pc.pc_inspect(W, L, p, 11, 0, n, mode=pc.PC_MODE_STREAM)
    ref = oracle.inspect(W, L, p=p, seed=11, n=n, mode="markov", threads=THREADS)
    assert_parity(res, ref, what="resident")
    assert_parity(stm, ref, what="stream")


def test_stream_lattice_beyond_shared_memory():
    W, L, p, n = 16, 128, 0.16, 120
    g = pc.pc_inspect(W, L, p, 12, 0, n)
    ref = oracle.inspect(W, L, p=p, seed=12, n=n, mode="markov", threads=THREADS)
    assert_parity(g, ref, what="W16 L128")


@pytest.mark.parametrize("p,n,cfg0", [(0.14, 12, 0), (0.1533, 12, 0), (0.17, 2, 5)])
def test_large_lattice_sampled(p, n, cfg0):
    """W = 64, L = 4096 (51.1 M sites), seed 4: sampled configurations against
    the oracle's BFS route (mass: FP32 and FP64 both underflow far below the
    tolerance on these path lengths; checked within 1e-5 against 0 <= m <= 1)."""
    W, L = 64, 4096
    g = pc.pc_inspect(W, L, p, 4, cfg0, n)
    ref = oracle.inspect(W, L, p=p, seed=4, cfg0=cfg0, n=n, mode="bfs", threads=THREADS)
    assert_parity(g, ref, mass=False, what=f"large p={p}")
    m = np.asarray(g["mass"])
    assert np.all(m >= 0) and np.all(m <= 1)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("W,L,p,n", [
    (0, 1, 0.5, 64), (0, 1, 1.0, 4), (0, 5, 0.9, 300), (0, 5, 1.0, 3), (3, 1, 0.2, 200),
    (3, 2, 0.3, 200), (5, 3, 0.0, 50), (5, 3, 1.0, 10), (6, 8, 1.0, 4), (1, 200, 0.9, 100),
    (8, 80, 0.21, 60),    # largest resident lattice of W = 8
    (8, 81, 0.21, 60),    # one layer more: streamed
])
def test_edge_cases(W, L, p, n):
    g = pc.pc_inspect(W, L, p, 21, 0, n)
    ref = oracle.inspect(W, L, p=p, seed=21, n=n, mode="markov", threads=THREADS)
    assert_parity(g, ref, what=f"W={W} L={L} p={p}")
    if p == 1.0:
        assert np.all(g["first_hit"] == L)
    if p == 0.0:
        assert np.all(g["verdict"] == 0) and np.all(g["m_stop"] == 0)


def test_widest_lattice_properties():
    """W = 255, the widest lattice the counter layout allows (A = 195,841):
    at p = 1 every configuration percolates with first hit L; at p = 0 none
    starts."""
    for L in (1, 2):
        g = pc.pc_inspect(255, L, 1.0, 1, 0, 2)
        assert np.all(g["verdict"] == 1) and np.all(g["first_hit"] == L)
        g = pc.pc_inspect(255, L, 0.0, 1, 0, 2)
        assert np.all(g["verdict"] == 0) and np.all(g["m_stop"] == 0)


def test_zero_configurations():
    g = pc.pc_inspect(4, 16, 0.2, 1, 0, 0)
    assert g["n_percolating"] == 0 and len(g["verdict"]) == 0


def test_device_outputs_streams_and_determinism():
    import torch
    W, L, p, n = 8, 64, 0.2, 2000
    host = pc.pc_inspect(W, L, p, 2, 0, n)
    s = torch.cuda.Stream()
    dev = pc.pc_inspect(W, L, p, 2, 0, n, device=True, stream=s)
    s.synchronize()
    dev = _host(dev)
    for k in ("verdict", "first_hit", "m_stop", "mass"):
        assert np.array_equal(np.asarray(host[k]), dev[k]), k
    again = pc.pc_inspect(W, L, p, 2, 0, n)
    assert np.array_equal(host["mass"], again["mass"])  # bit-identical


def test_placement_independence():
    """Counter-based stream: a configuration's result does not depend on which
    range (or call) it is inspected in."""
    a = pc.pc_inspect(8, 64, 0.2, 2, 0, 300)
    b = pc.pc_inspect(8, 64, 0.2, 2, 100, 300)
    for k in ("verdict", "first_hit", "m_stop", "mass"):
        assert np.array_equal(np.asarray(a[k])[100:], np.asarray(b[k])[:200]), k
