"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the printed
worked example of Fig. 2, an independent Philox implementation (PyTorch's
ATen engine, called as a library), the textbook cubic-coordinate definition
of the FCC lattice, closed forms (p = 0, p = 1, single-tube-wide fibre),
brute force over every configuration of a tiny lattice, a library
shortest-path routine (scipy), and invariants (Eq. (2) row sums, Appendix
Eq. (A.3) duality, 120-degree rotation symmetry, coupled monotonicity).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Philox4x32-10 and the occupancy stream (Sec. II.A sampling)
# ---------------------------------------------------------------------------

_ATEN_SRC = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>
extern "C" void aten_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  uint64_t seed = (uint64_t)key[0] | ((uint64_t)key[1] << 32);
  uint64_t sub = (uint64_t)ctr[2] | ((uint64_t)ctr[3] << 32);
  at::philox_engine e(seed, sub, 0);
  e.set_offset((uint64_t)ctr[0] | ((uint64_t)ctr[1] << 32));
  for (int i = 0; i < 4; ++i) out[i] = e();
}
"""


@pytest.fixture(scope="module")
def aten_philox():
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("ATen Philox engine header not available")
    d = tempfile.mkdtemp(prefix="aten_philox_")
    src = os.path.join(d, "p.cpp")
    so = os.path.join(d, "libp.so")
    with open(src, "w") as f:
        f.write(_ATEN_SRC)
    subprocess.run(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-I", inc, src, "-o", so],
                   check=True)
    lib = ctypes.CDLL(so)
    lib.aten_philox.argtypes = [ctypes.c_void_p] * 3

    def call(ctr, key):
        c = np.ascontiguousarray(ctr, np.uint32); k = np.ascontiguousarray(key, np.uint32)
        o = np.zeros(4, np.uint32)
        lib.aten_philox(c.ctypes.data, k.ctypes.data, o.ctypes.data)
        return o
    return call


def test_philox_matches_independent_engine(aten_philox):
    rng = np.random.default_rng(12345)
    cases = [([0, 0, 0, 0], [0, 0]), ([0xffffffff] * 4, [0xffffffff] * 2),
             ([1, 0, 0, 0], [0, 0]), ([0, 0, 0, 1], [0, 1])]
    for _ in range(300):
        cases.append((rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32),
                      rng.integers(0, 2**32, 2, dtype=np.uint64).astype(np.uint32)))
    for ctr, key in cases:
        assert np.array_equal(oracle.philox4x32_10(ctr, key), aten_philox(ctr, key)), (ctr, key)


def test_threshold_exact():
    for p in (0.0, 1.0, 0.5, 0.15, 0.1533, 0.2, 1e-12, 1 - 2**-40, 0.3):
        exact = math.floor(Fraction(p) * 2**32)
        assert oracle.threshold(p) == exact, p
    assert oracle.threshold(1.0) == 2**32


def test_occupancy_counter_layout(aten_philox):
    """site i of config c is metallic iff word (i & 3) of Philox(ctr = (i >> 2,
    c, W | L << 8, 0), key = seed halves) is below floor(p 2^32)."""
    W, L, p, seed = 2, 5, 0.37, 0x1234_5678_9ABC_DEF0
    A, N = oracle.lattice_info(W, L)
    occ = oracle.occupancy(W, L, p, seed, 7, 3)
    T = math.floor(Fraction(p) * 2**32)
    key = [seed & 0xffffffff, seed >> 32]
    for c in range(3):
        for i in range(N):
            w = aten_philox([i >> 2, 7 + c, W | (L << 8), 0], key)[i & 3]
            assert occ[c, i] == (1 if int(w) < T else 0)



def test_threshold_is_strict(aten_philox):
    """Metallic iff word < T (strict): choose p so that T equals site 0's word
    exactly (w / 2^32 is exact in double); site 0 is then insulating, and
    metallic at p = (w + 1) / 2^32."""
    W, L, seed = 1, 3, 77
    key = [seed & 0xffffffff, seed >> 32]
    w = int(aten_philox([0, 0, W | (L << 8), 0], key)[0])
    assert oracle.occupancy(W, L, w / 2**32, seed, 0, 1)[0, 0] == 0
    assert oracle.occupancy(W, L, (w + 1) / 2**32, seed, 0, 1)[0, 0] == 1

# ---------------------------------------------------------------------------
# Lattice (Sec. II.A, Fig. 1)
# ---------------------------------------------------------------------------

def test_column_count_and_paper_lattice_size():
    for W in range(0, 21):
        assert oracle.lattice_info(W, 1)[0] == 3 * W * (W + 1) + 1
    # Sec. III: "The largest lattice we inspected contains 2.6 million sites"
    A, N = oracle.lattice_info(46, 400)
    assert N == 2_594_800 and round(N / 1e6, 1) == 2.6


def _cubic(q, r, h):
    """Integer cubic coordinates of the FCC site at axial column (q, r), layer
    h: the linear map sending the three up-contacts (1,0,+1), (-1,1,+1),
    (0,-1,+1) to the FCC nearest neighbours (1,1,0), (0,1,1), (1,0,1)."""
    X = q - r + 2 * h
    Y = q + 2 * r + 2 * h
    Z = -2 * q - r + 2 * h
    assert X % 3 == 0 and Y % 3 == 0 and Z % 3 == 0
    return np.array([X // 3, Y // 3, Z // 3])


@pytest.mark.parametrize("W,L", [(0, 4), (1, 3), (2, 5), (4, 4), (6, 3)])
def test_adjacency_is_fcc_plus_end_contacts(W, L):
    """The oracle's neighbours are exactly the FCC nearest neighbours (cubic
    difference a permutation of (+-1, +-1, 0)) plus the two end contacts along
    <111> (difference +-(2, 2, 2)), restricted to the hexagonal fibre."""
    A, N = oracle.lattice_info(W, L)
    q, r, s = oracle.columns(W)
    nbr, cnt = oracle.adjacency(W, L)
    pos = {}
    coords = np.zeros((N, 3), np.int64)
    for i in range(N):
        a, t = i % A, i // A
        c = _cubic(int(q[a]), int(r[a]), 3 * t + int(s[a]))
        assert c.sum() % 2 == 0  # an FCC site
        coords[i] = c
        pos[tuple(c)] = i
    assert len(pos) == N  # injective
    nn = {tuple(v) for v in
          [(x, y, 0) for x in (-1, 1) for y in (-1, 1)] + [(x, 0, z) for x in (-1, 1) for z in (-1, 1)]
          + [(0, y, z) for y in (-1, 1) for z in (-1, 1)]}
    end = {(2, 2, 2), (-2, -2, -2)}
    for i in range(N):
        expect = set()
        for v in nn | end:
            j = pos.get(tuple(coords[i] + np.array(v)))
            if j is not None:
                expect.add(j)
        got = set(int(j) for j in nbr[i, :cnt[i]])
        assert got == expect, (i, got, expect)
        assert cnt[i] <= 14


def test_interior_coordination_14_and_symmetry():
    W, L = 4, 6
    A, N = oracle.lattice_info(W, L)
    q, r, s = oracle.columns(W)
    nbr, cnt = oracle.adjacency(W, L)
    for i in range(N):
        for j in nbr[i, :cnt[i]]:
            assert i in set(nbr[j, :cnt[j]])  # symmetric
        a, t = i % A, i // A
        interior = max(abs(q[a]), abs(r[a]), abs(q[a] + r[a])) <= W - 2 and 0 < t < L - 1
        if interior:
            assert cnt[i] == 14  # 12 side + 2 end contacts (Fig. 1(a))


def _rotation_perm(W, L):
    """Site permutation of the 120-degree rotation (q, r) -> (-q-r, q) about the
    central column; it keeps every sublattice and every tube index."""
    A, N = oracle.lattice_info(W, L)
    q, r, s = oracle.columns(W)
    idx = {(int(q[a]), int(r[a])): a for a in range(A)}
    col = np.array([idx[(-int(q[a]) - int(r[a]), int(q[a]))] for a in range(A)])
    assert all(s[col[a]] == s[a] for a in range(A))
    return np.concatenate([col + t * A for t in range(L)])


def test_rotation_is_an_automorphism():
    W, L = 3, 4
    perm = _rotation_perm(W, L)
    nbr, cnt = oracle.adjacency(W, L)
    for i in range(len(perm)):
        a = set(int(perm[j]) for j in nbr[i, :cnt[i]])
        b = set(int(j) for j in nbr[perm[i], :cnt[perm[i]]])
        assert a == b


# ---------------------------------------------------------------------------
# Markov inspection (Sec. II.B, Eqs. (1)-(4), Appendix)
# ---------------------------------------------------------------------------

def _load_fig2():
    rows = []
    with open(os.path.join(GOLDEN, "fig2_transition_matrix.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(Fraction(x)) for x in line.split()])
    return np.array(rows)


def test_fig2_worked_example():
    P = _load_fig2()
    assert P.shape == (7, 7)
    assert np.allclose(P.sum(axis=1), 1.0)  # Eq. (2): rows sum to one
    f = oracle.first_passage_dense(P, j0=6, i0=0, mmax=12)
    assert np.all(f[:5] == 0.0)              # m < 6: zero (Fig. 2)
    assert f[5] > 0.0                        # m = 6: positive (Fig. 2)
    # the only 6-step walk 1 -> 7 goes straight along: 1 * (1/2)^5
    assert f[5] == pytest.approx(1 / 32, rel=1e-15)
    n_bonds = int(np.count_nonzero(np.triu(P + P.T)))
    assert n_bonds == 6                      # tau_{1->7} = N_b = 6 (Sec. II.B)
    # tube 5 insulating: the remaining tubes 1-4 and 6-7 form two paths
    keep = [0, 1, 2, 3, 5, 6]
    adj = (P[np.ix_(keep, keep)] > 0).astype(float)
    Pc = adj / adj.sum(axis=1, keepdims=True)
    g = oracle.first_passage_dense(Pc, j0=5, i0=0, mmax=60)
    assert np.all(g == 0.0)                  # tau = infinity


@pytest.mark.parametrize("W,L", [(0, 1), (0, 6), (2, 1), (2, 7), (4, 16)])
def test_p0_and_p1(W, L):
    r0 = oracle.inspect(W, L, p=0.0, seed=3, n=20, mode="markov")
    assert np.all(r0["verdict"] == 0) and np.all(r0["m_stop"] == 0)
    r1 = oracle.inspect(W, L, p=1.0, seed=3, n=5, mode="markov")
    # each step changes the layer height by at most 3 = one tube period
    assert np.all(r1["verdict"] == 1) and np.all(r1["first_hit"] == L)


@pytest.mark.parametrize("L", [1, 2, 3, 8, 30])
def test_single_tube_wide_fibre(L):
    """W = 0: the fibre is one column; it percolates iff all L tubes are
    metallic, the walk must go straight up, so a_L = 2^-(L-1) (L >= 2: the
    bottom tube has one contact, the others two, the top one counting the
    detector), 1 for L = 1."""
    r = oracle.inspect(0, L, p=1.0, seed=1, n=1, mode="markov")
    assert r["first_hit"][0] == L
    assert r["mass"][0] == pytest.approx(1.0 if L == 1 else 2.0 ** -(L - 1), rel=1e-14)
    occ = oracle.occupancy(0, L, 0.8, 11, 0, 400)
    r = oracle.inspect(0, L, occ=occ, mode="markov")
    for c in range(400):
        col = occ[c]
        assert r["verdict"][c] == int(col.all())
        if not col[0]:
            assert r["m_stop"][c] == 0
        elif not col.all():
            k = int(np.argmin(col))          # first insulating tube
            assert r["m_stop"][c] == k


@pytest.mark.parametrize("W,L,seed,spread", [(3, 12, 5, None), (8, 30, 6, None), (16, 40, 7, 6)])
def test_wire_first_passage_closed_form(W, L, seed, spread):
    """A single induced path of metallic sites from t = 0 to t = L-1 (the
    parity tests' wires): the walk can only follow it, so the first hit is at
    m = number of path sites and the absorbed mass is 2^-(sites-1) exactly
    (deg 1 at the start, 2 inside, 2 at the end with the detector edge).
    The path is built from the geometric contact table, and verified here to
    be induced by BFS of the oracle itself."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import _wires
    occ, sites = _wires.wire_occupancies(W, L, 6, seed, spread=spread)
    nbr, cnt = oracle.adjacency(W, L)
    for c in range(occ.shape[0]):
        on = np.flatnonzero(occ[c])
        # every wire site has at most 2 metallic contacts (induced path)
        deg = [int(sum(occ[c][j] for j in nbr[i, :cnt[i]])) for i in on]
        assert max(deg) <= 2 and sorted(deg).count(1) == (2 if len(on) > 1 else 0)
    r = oracle.inspect(W, L, occ=occ, mode="markov")
    b = oracle.inspect(W, L, occ=occ, mode="bfs")
    assert np.array_equal(r["first_hit"], sites) and np.array_equal(b["first_hit"], sites)
    assert np.array_equal(r["mass"], 2.0 ** -(sites - 1.0))


def _all_patterns(N):
    k = np.arange(2**N, dtype=np.uint32)
    return ((k[:, None] >> np.arange(N, dtype=np.uint32)) & 1).astype(np.uint8)


def test_brute_force_all_configurations():
    """Every one of the 2^14 configurations of W = 1, L = 2: Markov, BFS and
    union-find agree; running the recursion on to N_max finds no late hit."""
    W, L = 1, 2
    A, N = oracle.lattice_info(W, L)
    assert N == 14
    occ = _all_patterns(N)
    mk = oracle.inspect(W, L, occ=occ, mode="markov_full", stats=True)
    bf = oracle.inspect(W, L, occ=occ, mode="bfs")
    uf = oracle.inspect(W, L, occ=occ, mode="unionfind")
    assert np.array_equal(mk["verdict"], bf["verdict"])
    assert np.array_equal(mk["verdict"], uf["verdict"])
    assert np.array_equal(mk["first_hit"], bf["first_hit"])
    assert np.array_equal(mk["m_stop"], bf["m_stop"])
    assert np.all(mk["stats"]["nmax_ok"] == 1)
    assert 0 < mk["verdict"].sum() < len(occ)


def test_monte_carlo_matches_exact_polynomial():
    """Pi(p) = sum over percolating configurations of p^k (1-p)^(N-k); the
    stream's Monte Carlo estimate must agree within sampling error."""
    W, L = 1, 2
    A, N = oracle.lattice_info(W, L)
    occ = _all_patterns(N)
    perc = oracle.inspect(W, L, occ=occ, mode="unionfind")["verdict"].astype(bool)
    k = occ.sum(axis=1)
    n = 20000
    for p in (0.3, 0.55, 0.8):
        exact = float(np.sum(np.where(perc, p ** k * (1 - p) ** (N - k), 0.0)))
        mc = oracle.inspect(W, L, p=p, seed=99, n=n, mode="bfs")["verdict"].mean()
        sigma = math.sqrt(exact * (1 - exact) / n)
        assert abs(mc - exact) < 5 * sigma + 1e-12, (p, mc, exact)


def test_coupled_monotonicity():
    """p is not part of the counter: each site keeps its uniform word across
    p, so occupancy and verdicts are monotone in p per configuration."""
    W, L, seed = 3, 6, 5
    prev_occ = prev_v = None
    for p in np.linspace(0.1, 0.6, 11):
        occ = oracle.occupancy(W, L, p, seed, 0, 300)
        v = oracle.inspect(W, L, p=p, seed=seed, n=300, mode="bfs")["verdict"]
        if prev_occ is not None:
            assert np.all(occ >= prev_occ) and np.all(v >= prev_v)
        prev_occ, prev_v = occ, v


def test_forward_backward_duality():
    """Appendix Eq. (A.3): the backward recursion f^(m) = ^(j1)P f^(m-1) and
    the forward propagation of mu_0 give the same first-passage probability
    a_m = mu_0^T f^(m); a_m vanishes before first_hit and equals the reported
    mass at first_hit."""
    W, L = 2, 5
    occ = oracle.occupancy(W, L, 0.55, 21, 0, 40)
    r = oracle.inspect(W, L, occ=occ, mode="markov")
    for c in range(40):
        fw, bw = oracle.first_passage(W, L, occ[c], 25)
        assert np.allclose(fw, bw, rtol=1e-12, atol=1e-300)
        if r["verdict"][c]:
            m = r["first_hit"][c]
            assert np.all(fw[: m - 1] == 0.0) and fw[m - 1] > 0
            assert fw[m - 1] == pytest.approx(r["mass"][c], rel=1e-12)
        else:
            assert np.all(fw == 0.0)


def test_mass_conservation_and_nmax():
    """Rows of P sum to one (Eq. (2)): mass left + absorbed + dropped at
    isolated sites = 1; and m_stop <= N_max = min(N_b, Np) + 1 (Sec. II.B)."""
    r = oracle.inspect(4, 16, p=0.3, seed=8, n=300, mode="markov_full", stats=True)
    st = r["stats"]
    has = st["n0"] > 0
    total = st["residual"] + st["absorbed"] + st["dropped"]
    assert np.allclose(total[has], 1.0, atol=1e-12)
    assert np.all(st["nmax_ok"] == 1)


def test_fp64_nonzero_rule_agrees_with_support():
    """Sec. II.B stops when the detector probability becomes non-zero; on
    lattices small enough that FP64 cannot underflow, that rule and the exact
    support rule give the same first hit."""
    r = oracle.inspect(3, 10, p=0.45, seed=4, n=300, mode="markov", stats=True)
    fp = r["stats"]["fp_first_nonzero"].astype(int)
    fh = r["first_hit"]
    assert np.array_equal(np.where(r["verdict"] == 1, fh, -1), fp)
    assert r["verdict"].sum() > 20


def test_first_hit_is_shortest_spanning_path():
    """Sec. II.B: the first hit gives the length of the shortest spanning path.
    Checked against scipy's breadth-first shortest paths."""
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    W, L = 3, 8
    A, N = oracle.lattice_info(W, L)
    nbr, cnt = oracle.adjacency(W, L)
    occ = oracle.occupancy(W, L, 0.5, 17, 0, 60)
    r = oracle.inspect(W, L, occ=occ, mode="markov")
    rows = np.repeat(np.arange(N), cnt)
    cols = np.concatenate([nbr[i, :cnt[i]] for i in range(N)])
    for c in range(60):
        o = occ[c].astype(bool)
        keep = o[rows] & o[cols]
        # super-source joined to the metallic sites of t = 0
        src = np.flatnonzero(o[:A])
        rr = np.concatenate([rows[keep], np.full(len(src), N)])
        cc = np.concatenate([cols[keep], src])
        g = sp.csr_matrix((np.ones(len(rr)), (rr, cc)), shape=(N + 1, N + 1))
        d = csg.shortest_path(g, method="D", unweighted=True, indices=N)
        end = d[(L - 1) * A: L * A][o[(L - 1) * A: L * A]]
        if len(src) and np.isfinite(end).any():
            assert r["verdict"][c] == 1
            assert r["first_hit"][c] == int(end.min())  # = (path length) + 1
        else:
            assert r["verdict"][c] == 0


def test_rotation_invariance():
    W, L = 3, 7
    perm = _rotation_perm(W, L)
    occ = oracle.occupancy(W, L, 0.5, 31, 0, 80)
    rot = np.zeros_like(occ)
    rot[:, perm] = occ           # site i moves to perm[i]
    a = oracle.inspect(W, L, occ=occ, mode="markov")
    b = oracle.inspect(W, L, occ=rot, mode="markov")
    for k in ("verdict", "first_hit", "m_stop"):
        assert np.array_equal(a[k], b[k])
    assert np.allclose(a["mass"], b["mass"], rtol=1e-12, atol=0)


def test_single_layer_fibre():
    """L = 1: the start surface is the end surface; the first hit is m = 1 and
    a_1 = (1/n0) sum over metallic sites of 1/deg (deg counts the detector)."""
    W = 2
    A, N = oracle.lattice_info(W, 1)
    nbr, cnt = oracle.adjacency(W, 1)
    occ = oracle.occupancy(W, 1, 0.5, 2, 0, 50)
    r = oracle.inspect(W, 1, occ=occ, mode="markov")
    for c in range(50):
        o = occ[c]
        if not o.any():
            assert r["verdict"][c] == 0 and r["m_stop"][c] == 0
            continue
        assert r["verdict"][c] == 1 and r["first_hit"][c] == 1
        n0 = int(o.sum())
        deg = [1 + int(o[nbr[i, :cnt[i]]].sum()) for i in range(N) if o[i]]
        assert r["mass"][c] == pytest.approx(sum(1.0 / d for d in deg) / n0, rel=1e-14)


def test_site_update_accounting():
    """sum_{m=1}^{M} min(m+1, L) written out as a loop."""
    for L in (1, 2, 5, 64):
        for M in range(0, 80):
            brute = sum(min(m + 1, L) for m in range(1, M + 1))
            v = [0]; fh = [-1]; ms = [M]
            assert oracle.site_updates(1, L, v, fh, ms) == brute
            if M >= 1:
                assert oracle.site_updates(3, L, [1], [M + 1], [M + 1]) == 3 * brute


# ---------------------------------------------------------------------------
# fixed-count sample space (Sec. II.A: a random permutation puts exactly Np
# of the N sites metallic)
# ---------------------------------------------------------------------------

def test_fixed_count_has_exactly_np_sites():
    for W, L, Np in [(2, 5, 0), (2, 5, 37), (2, 5, 95), (3, 7, 100)]:
        _, N = oracle.lattice_info(W, L)
        occ = oracle.occupancy_fixed(W, L, min(Np, N), seed=5, cfg0=0, n=20)
        assert np.all(occ.sum(axis=1) == min(Np, N))


def test_fixed_count_couples_with_bernoulli():
    # the Np sites with the smallest words are exactly the sites below the
    # Bernoulli threshold whenever Np is the Bernoulli count
    W, L, p, seed = 3, 9, 0.3, 17
    bern = oracle.occupancy(W, L, p, seed, 0, 50)
    for c in range(50):
        Np = int(bern[c].sum())
        fixed = oracle.occupancy_fixed(W, L, Np, seed, c, 1)[0]
        assert np.array_equal(fixed, bern[c])


def test_fixed_count_is_uniform_over_subsets():
    # W = 1, L = 1: N = 7 sites, Np = 3 -> C(7, 3) = 35 subsets, equally likely
    from math import comb
    n = 14000
    occ = oracle.occupancy_fixed(1, 1, 3, seed=23, cfg0=0, n=n)
    codes = (occ.astype(np.int64) << np.arange(7)).sum(axis=1)
    _, counts = np.unique(codes, return_counts=True)
    assert counts.size == comb(7, 3)
    expected = n / comb(7, 3)
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < 70.0  # 34 degrees of freedom: P(chi2 > 70) < 1e-3


# ---------------------------------------------------------------------------
# The lazy walk of the self-loop remark (Sec. II.B): staying put with
# probability s does not change percolation.  Under s I + (1 - s) P the first
# passage at the shortest spanning length needs a move at every step, so it is
# (1 - s)^m times the plain one, and the probability of ever being absorbed is
# unchanged.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("s", [0.25, 0.5, 0.9])
def test_lazy_walk_on_fig2(s):
    P = _load_fig2()
    Ps = s * np.eye(7) + (1 - s) * P
    f = oracle.first_passage_dense(Ps, j0=6, i0=0, mmax=int(1500 / (1 - s)))
    assert np.all(f[:5] == 0.0)
    assert f[5] == pytest.approx((1 - s) ** 6 / 32, rel=1e-13)
    assert f.sum() == pytest.approx(1.0, abs=1e-9)  # the chain is connected


@pytest.mark.parametrize("s", [0.0, 0.25, 0.5, 0.9])
def test_lazy_walk_keeps_first_hit_and_scales_its_mass(s):
    W, L = 2, 5
    occ = oracle.occupancy(W, L, 0.55, 21, 0, 40)
    r = oracle.inspect(W, L, occ=occ, mode="markov")
    for c in range(40):
        plain, _ = oracle.first_passage(W, L, occ[c], 25)
        lazy = oracle.first_passage_lazy(W, L, occ[c], 25, s)
        if s == 0.0:
            assert np.array_equal(lazy, plain)
        if r["verdict"][c]:
            m = r["first_hit"][c]
            assert np.all(lazy[: m - 1] == 0.0) and lazy[m - 1] > 0
            assert lazy[m - 1] == pytest.approx((1 - s) ** m * r["mass"][c], rel=1e-12)
        else:
            assert np.all(lazy == 0.0)


def test_lazy_walk_absorbs_the_same_total():
    W, L = 1, 4
    occ = oracle.occupancy(W, L, 0.7, 5, 0, 12)
    for c in range(12):
        plain, _ = oracle.first_passage(W, L, occ[c], 3000)
        lazy = oracle.first_passage_lazy(W, L, occ[c], 6000, 0.5)
        assert lazy.sum() == pytest.approx(plain.sum(), abs=1e-10)


def test_lazy_walk_rejects_hold_outside_unit_interval():
    occ = oracle.occupancy(1, 3, 0.5, 1, 0, 1)[0]
    for bad in (-0.1, 1.0, float("nan")):
        with pytest.raises(RuntimeError):
            oracle.first_passage_lazy(1, 3, occ, 5, bad)
