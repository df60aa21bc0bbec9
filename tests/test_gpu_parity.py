"""GPU parity: libpercol (through its C ABI) against the CPU oracle.

Verdicts, first_hit and m_stop are compared bit-exact on every configuration.
The FP32 detector mass is compared with the oracle's FP64 mass twice: within
the absolute tolerance 1e-5, and, wherever the FP64 mass exceeds 1e-30,
within the relative bound ``mass_rel_bound`` derived from the kernels'
summation order (below).  Occupancy bits are compared bit-exact.
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

# Relative bound of the FP32 mass.  All quantities are non-negative, so a
# rounding error of each operation, relative u = 2^-24, stays relative through
# every later sum and product.  The start value nu_0 = RN(RN(1/deg) RN(1/n0))
# carries 3u.  One step sums 14 neighbour values in an addition tree of depth
# at most 5 and multiplies by RN(1/deg): 7u per step, so nu after step m
# carries (3 + 7m)u.  The mass at first_hit = fh sums the end-layer entries of
# nu_{fh-1} over the P plane positions in one CTA: a serial sum of at most
# ceil(P / 32) terms per thread (CTAs have >= 32 threads) and then two warp
# trees of depth 5.  Second-order terms are covered by the factor 1.01.
# Below 1e-30 the relative check is skipped: without flush-to-zero every
# subnormal operation errs by at most 2^-150 absolute, and the ~10^8
# operations behind one mass stay below 1e-37, 1e-7 of such a mass.
U24 = 2.0 ** -24
MASS_REL_FLOOR = 1e-30
_PLANE = {}


def plane_entries(W):
    if W not in _PLANE:
        _PLANE[W] = pc.pc_lattice_layout(W)["P"]
    return _PLANE[W]


def mass_rel_bound(first_hit, W):
    fh = np.maximum(np.asarray(first_hit, np.int64), 1)
    return 1.01 * (3 + 7 * (fh - 1) + (plane_entries(W) + 31) // 32 + 10) * U24


def mass_rel_check(gpu, ref, W, what=""):
    """Element-wise relative check where the FP64 mass is above the floor;
    returns (configurations checked, largest relative error)."""
    mg = np.asarray(gpu["mass"]).astype(np.float64)
    mr = np.asarray(ref["mass"], np.float64)
    sel = mr > MASS_REL_FLOOR
    if not sel.any():
        return 0, 0.0
    rel = np.abs(mg[sel] - mr[sel]) / mr[sel]
    tol = mass_rel_bound(np.asarray(ref["first_hit"])[sel], W)
    bad = np.flatnonzero(rel > tol)
    assert bad.size == 0, f"{what}: relative mass error {rel[bad[:5]]} above {tol[bad[:5]]}"
    return int(sel.sum()), float(rel.max())


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


def assert_parity(gpu, ref, mass=True, what="", W=None):
    """Bit-exact verdict, first_hit, m_stop; mass within 1e-5 absolute and,
    with the lattice's W given, within the relative bound above the floor."""
    v = np.asarray(gpu["verdict"]).astype(np.int32)
    assert np.array_equal(v, ref["verdict"]), f"{what}: verdicts differ at {np.flatnonzero(v != ref['verdict'])[:10]}"
    assert np.array_equal(np.asarray(gpu["first_hit"]), ref["first_hit"]), what
    assert np.array_equal(np.asarray(gpu["m_stop"]), ref["m_stop"]), what
    if mass:
        err = np.abs(np.asarray(gpu["mass"]).astype(np.float64) - ref["mass"])
        assert err.max(initial=0.0) <= MASS_TOL, f"{what}: mass error {err.max()}"
        if W is not None:
            return mass_rel_check(gpu, ref, W, what)
    return 0, 0.0


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
    assert_parity(g, ref, what="tiny", W=W)
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
        assert_parity(g, ref, what=f"p={p}", W=W)
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
    assert_parity(g, ref, what="brute force", W=W)


def test_random_explicit_occupancies_ragged():
    import torch
    rng = np.random.default_rng(3)
    for W, L in [(2, 9), (5, 11), (7, 33)]:
        A, N = oracle.lattice_info(W, L)
        occ = (rng.random((200, N)) < 0.45).astype(np.uint8)
        bits = torch.from_numpy(oracle.pack_bits(occ).view(np.int32)).cuda()
        g = pc.pc_inspect_occupancy(W, L, bits)
        ref = oracle.inspect(W, L, occ=occ, mode="markov", threads=THREADS)
        assert_parity(g, ref, what=f"explicit W={W} L={L}", W=W)


# ---------------------------------------------------------------------------
# streamed solver
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("W,L,p,n", [(4, 16, 0.3, 300), (8, 64, 0.19, 400), (3, 40, 0.45, 200)])
def test_stream_mode_matches_resident_and_oracle(W, L, p, n):
    res = pc.pc_inspect(W, L, p, 11, 0, n, mode=pc.PC_MODE_RESIDENT)
    stm = pc.pc_inspect(W, L, p, 11, 0, n, mode=pc.PC_MODE_STREAM)
    ref = oracle.inspect(W, L, p=p, seed=11, n=n, mode="markov", threads=THREADS)
    assert_parity(res, ref, what="resident", W=W)
    assert_parity(stm, ref, what="stream", W=W)


def test_stream_lattice_beyond_shared_memory():
    W, L, p, n = 16, 128, 0.16, 120
    g = pc.pc_inspect(W, L, p, 12, 0, n)
    ref = oracle.inspect(W, L, p=p, seed=12, n=n, mode="markov", threads=THREADS)
    assert_parity(g, ref, what="W16 L128", W=W)


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
# FP32 mass, element by element, on both solvers
# ---------------------------------------------------------------------------

def _resident_or_none(W, L, p, seed, n):
    """pc_inspect in resident mode, or None when the state exceeds shared memory."""
    try:
        return pc.pc_inspect(W, L, p, seed, 0, n, mode=pc.PC_MODE_RESIDENT)
    except pc.PercolError as e:
        if e.status == pc.PC_ERR_OOM:
            return None
        raise


MASS_CASES = [(W, L, p) for W in (16, 32, 64) for L in (1, 4, 8, 16, 24) for p in (0.3, 0.6, 0.9)]


@pytest.mark.parametrize("W,L,p", MASS_CASES)
def test_mass_relative_both_solvers(W, L, p):
    """Eqs. (3)-(4): the FP32 mass of every configuration within the relative
    bound of the FP64 oracle.  Lattices of 2 (W = 16) to 17 (W = 64)
    256-strip FP chunks, every plane cycled through the streamed solver's
    ring; at these lengths every oracle mass is above the floor, so no
    configuration escapes the relative check."""
    n, seed = {16: 128, 32: 96, 64: 48}[W], 31
    ref = oracle.inspect(W, L, p=p, seed=seed, n=n, mode="markov", threads=THREADS)
    runs = [("stream", pc.pc_inspect(W, L, p, seed, 0, n, mode=pc.PC_MODE_STREAM))]
    res = _resident_or_none(W, L, p, seed, n)
    if res is not None:
        runs.append(("resident", res))
    for name, g in runs:
        k, mx = assert_parity(g, ref, what=f"{name} W={W} L={L} p={p}", W=W)
        assert k == n, f"{name}: only {k} of {n} masses above the floor"
        print(f"mass-rel {name} W={W} L={L} p={p}: {k} configurations, max rel {mx:.3e}, "
              f"bound at max first_hit {mass_rel_bound(ref['first_hit'].max(), W):.3e}")


@pytest.mark.parametrize("mode", [pc.PC_MODE_STREAM, pc.PC_MODE_RESIDENT])
@pytest.mark.parametrize("L", [1, 2, 5, 64, 127, 128, 129, 130, 150])
def test_mass_single_column_closed_form(L, mode):
    """W = 0, p = 1: a single wire of L tubes; the mass at first_hit = L is
    exactly 2^-(L-1) (Sec. II.B walk with the detector edge), down to 2^-149.
    L > 128 puts layers into a second 128-layer FP unit of the streamed
    solver."""
    g = pc.pc_inspect(0, L, 1.0, 3, 0, 4, mode=mode)
    assert np.all(g["verdict"] == 1) and np.all(g["first_hit"] == L)
    assert np.all(g["mass"].astype(np.float64) == 2.0 ** -(L - 1)), g["mass"]


def _wire_case(W, L, n, seed, spread, mode):
    import torch
    import _wires
    occ, sites = _wires.wire_occupancies(W, L, n, seed, spread=spread)
    bits = torch.from_numpy(oracle.pack_bits(occ).view(np.int32)).cuda()
    g = pc.pc_inspect_occupancy(W, L, bits, mode=mode)
    ref = oracle.inspect(W, L, occ=occ, mode="markov", threads=THREADS)
    assert_parity(g, ref, what=f"wires W={W} L={L}", W=W)
    # closed form on both sides, exact: first hit = sites, mass = 2^-(sites-1)
    assert np.array_equal(ref["first_hit"], sites) and np.array_equal(g["first_hit"], sites)
    assert np.array_equal(ref["mass"], 2.0 ** -(sites - 1.0))
    assert np.array_equal(g["mass"].astype(np.float64), 2.0 ** -(sites - 1.0))
    return sites


def test_mass_wires_across_the_wide_lattice():
    """W = 64, L = 60: single induced paths of metallic sites steered through
    random waypoints anywhere in the hexagon, so they cross many of the 17
    strip chunks and rows of the streamed solver's FP units.  The masses are
    2^-75 .. 2^-149, far beyond where random configurations keep any FP32
    mass, and both sides must give them exactly."""
    sites = _wire_case(64, 60, 16, 41, None, pc.PC_MODE_STREAM)
    assert sites.min() > 60


def test_mass_wires_into_the_second_fp_unit():
    """W = 64, L = 140: wires that climb past layer 128 (a second FP unit
    along the fibre), mass 2^-139 .. 2^-149 (FP32 subnormals, still exact)."""
    sites = _wire_case(64, 140, 8, 43, 4, pc.PC_MODE_STREAM)
    assert sites.max() <= 150


def test_mass_wires_resident():
    """Wires on the largest resident lattice of W = 8 (L = 74), across the
    hexagon and up the fibre, through the resident solver."""
    _wire_case(8, 74, 16, 47, None, pc.PC_MODE_RESIDENT)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("W,L,p,n", [
    (0, 1, 0.5, 64), (0, 1, 1.0, 4), (0, 5, 0.9, 300), (0, 5, 1.0, 3), (3, 1, 0.2, 200),
    (3, 2, 0.3, 200), (5, 3, 0.0, 50), (5, 3, 1.0, 10), (6, 8, 1.0, 4), (1, 200, 0.9, 100),
    (8, 74, 0.21, 60),    # largest resident lattice of W = 8
    (8, 75, 0.21, 60),    # one layer more: streamed
])
def test_edge_cases(W, L, p, n):
    g = pc.pc_inspect(W, L, p, 21, 0, n)
    ref = oracle.inspect(W, L, p=p, seed=21, n=n, mode="markov", threads=THREADS)
    assert_parity(g, ref, what=f"W={W} L={L} p={p}", W=W)
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
