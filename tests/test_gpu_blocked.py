"""The verdict-only solver with temporal blocking (PC_BITS_ONLY on the streamed
path): 32 steps of the exact reached-set propagation per visit of a slab of
word rows, the lattice's whole cross-section held in the shared memory of one
thread-block cluster (Sec. II.B: the reached set alone decides percolation).

Verdicts, first_hit and m_stop must equal the BFS oracle's bit for bit on
lattices that take clusters of 1, 2, 4 and 16 CTAs, several slabs per pass,
ragged fibre lengths and the degenerate cases; and the step-synchronous
solver's (PC_BITS_STEPWISE=1) at the benchmark's full size, W = 64,
L = 4096."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
import paper_1401_2130_gb300 as pc

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1
STREAM_BITS = pc.PC_MODE_STREAM | pc.PC_BITS_ONLY


def _check(g, ref, what):
    assert np.array_equal(np.asarray(g["verdict"]).astype(np.int32), np.asarray(ref["verdict"]).astype(np.int32)), what
    assert np.array_equal(np.asarray(g["first_hit"]), np.asarray(ref["first_hit"])), what
    assert np.array_equal(np.asarray(g["m_stop"]), np.asarray(ref["m_stop"])), what


def _stepwise(*args, **kw):
    os.environ["PC_BITS_STEPWISE"] = "1"
    try:
        return pc.pc_inspect(*args, **kw)
    finally:
        del os.environ["PC_BITS_STEPWISE"]


@pytest.mark.parametrize("W,cs", [(0, 1), (12, 1), (15, 1), (16, 2), (32, 4), (64, 16)])
def test_cluster_shape(W, cs):
    """Columns per CTA = ceil(A / cluster size) <= 800 (one per thread): the
    smallest cluster that holds the cross-section (A = 3W(W+1)+1 columns)."""
    s = pc.pc_bits_blocked_shape(W)
    assert s is not None, W
    A = 3 * W * (W + 1) + 1
    assert s["cluster_size"] == cs
    assert s["columns_per_cta"] == -(-A // cs) <= 800
    assert s["slab_rows"] % 4 == 0 and 12 <= s["slab_rows"] <= 36 and s["clusters"] >= 1


@pytest.mark.parametrize("W,L,p,seed,cfg0,n", [
    (20, 2000, 0.19, 5, 0, 48),    # 2 CTAs per cluster, 3 slabs, L not a multiple of 32
    (32, 1500, 0.17, 6, 10, 24),   # 4 CTAs, 3 slabs
    (64, 1500, 0.16, 4, 0, 6),     # 16 CTAs
    (12, 2100, 0.2, 3, 0, 64),     # one CTA, 3 slabs
    (20, 32, 0.3, 1, 0, 200),      # one word row exactly
    (20, 33, 0.3, 1, 0, 200),      # a second row of one tube
    (20, 65, 0.25, 8, 3, 200),     # three rows, the last of one tube
    (20, 64, 1.0, 1, 0, 4),        # every site metallic: straight runs
    (20, 100, 0.0, 1, 0, 4),       # nothing metallic: n0 = 0
    (20, 1, 0.5, 2, 0, 64),        # L = 1
    (0, 3000, 0.995, 4, 0, 32),    # one tube: stops at the first empty site
])
def test_blocked_equals_bfs_oracle(W, L, p, seed, cfg0, n):
    assert pc.pc_bits_blocked_shape(W) is not None
    g = pc.pc_inspect(W, L, p, seed, cfg0, n, mode=pc.PC_MODE_STREAM, bits_only=True)
    ref = oracle.inspect(W, L, p=p, seed=seed, cfg0=cfg0, n=n, mode="bfs", threads=THREADS)
    _check(g, ref, (W, L, p))
    assert g["n_percolating"] == int(ref["verdict"].sum())
    assert not np.any(g["mass"])
    if L >= 1500:
        # some configuration runs for several passes
        steps = np.where(ref["verdict"] != 0, ref["first_hit"] - 1, ref["m_stop"])
        assert steps.max() > 64, steps.max()


def test_blocked_equals_stepwise_at_full_size():
    """The benchmark's lattice (W = 64, L = 4096: 51.1 M sites) at the three
    benchmark probabilities: the blocked and the step-synchronous solvers
    agree on every configuration; one configuration per p is checked against
    the BFS oracle as well."""
    W, L, seed, n = 64, 4096, 4, 4
    for p in (0.14, 0.1533, 0.17):
        g = pc.pc_inspect(W, L, p, seed, 0, n, mode=pc.PC_MODE_STREAM, bits_only=True)
        s = _stepwise(W, L, p, seed, 0, n, mode=pc.PC_MODE_STREAM, bits_only=True)
        _check(g, s, p)
        ref = oracle.inspect(W, L, p=p, seed=seed, cfg0=1, n=1, mode="bfs", threads=THREADS)
        _check({k: np.asarray(v)[1:2] for k, v in g.items() if k in ("verdict", "first_hit", "m_stop")}, ref, p)


def test_blocked_matches_the_full_inspection():
    """The FP32 inspection's verdicts and step counts are the same numbers."""
    W, L, p, seed, n = 32, 600, 0.18, 9, 32
    g = pc.pc_inspect(W, L, p, seed, 0, n, mode=pc.PC_MODE_STREAM, bits_only=True)
    full = pc.pc_inspect(W, L, p, seed, 0, n, mode=pc.PC_MODE_STREAM)
    _check(g, full, "full")


def test_blocked_slots_are_refilled():
    """More configurations than slots: finished slots take new ones, and the
    stale rows a previous configuration left in a slot are never read."""
    W, L, p, seed, n = 20, 300, 0.2, 13, 700
    g = pc.pc_inspect(W, L, p, seed, 0, n, mode=pc.PC_MODE_STREAM, bits_only=True)
    s = _stepwise(W, L, p, seed, 0, n, mode=pc.PC_MODE_STREAM, bits_only=True)
    _check(g, s, "refill")
    ref = oracle.inspect(W, L, p=p, seed=seed, n=n, mode="bfs", threads=THREADS)
    _check(g, ref, "refill oracle")


def test_blocked_fixed_count_occupancy():
    """Caller occupancies (the fixed-count sample space of Sec. II.A) through
    the blocked solver."""
    W, L, seed, n = 20, 400, 3, 24
    _, N = oracle.lattice_info(W, L)
    Np = int(round(0.19 * N))
    bits = pc.pc_occupancy_fixed(W, L, Np, seed, 0, n)
    g = pc.pc_inspect_occupancy(W, L, bits, mode=STREAM_BITS)
    occ = oracle.occupancy_fixed(W, L, Np, seed, 0, n)
    ref = oracle.inspect(W, L, occ=occ, mode="bfs", threads=THREADS)
    _check(g, ref, "fixed count")


def test_blocked_in_verdict_only_batches():
    """pc_batch_run with PC_BITS_ONLY: the streamed queries that a cluster
    holds run on the blocked solver (solver "blocked"), the others as before;
    results equal the oracle's and the step-synchronous solver's.  PC_ASYNC
    batches keep the step-synchronous slots, with the same results."""
    import torch
    specs = [(4, 8, 0.2, 3, 0, 400), (20, 400, 0.19, 3, 5, 64), (32, 300, 0.17, 4, 0, 24),
             (12, 200, 0.17, 3, 0, 64), (8, 64, 0.18, 3, 100, 300)]
    outs, res = pc.pc_batch_run(specs, bits_only=True)
    for sp, o, r in zip(specs, outs, res):
        W, L, p, seed, b, n = sp
        ref = oracle.inspect(W, L, p=p, seed=seed, cfg0=b, n=n, mode="bfs", threads=THREADS)
        _check(o, ref, sp)
        assert r["n_percolating"] == int(ref["verdict"].sum())
        step = _stepwise(W, L, p, seed, b, n, bits_only=True)
        _check(o, step, (sp, "step-synchronous"))
        want = "resident" if (W, L) in ((4, 8), (8, 64)) else "blocked"
        assert r["solver"] == want, (sp, r["solver"])
    # asynchronous batch: device outputs, step-synchronous slots, same results
    outs_a, _ = pc.pc_batch_run(specs, bits_only=True, device=True, async_=True)
    torch.cuda.synchronize()
    for sp, o, oa in zip(specs, outs, outs_a):
        _check({k: v.cpu().numpy() for k, v in oa.items() if k in ("verdict", "first_hit", "m_stop")}, o, sp)


def test_blocked_device_outputs():
    """PC_OUT_DEVICE: the passes run inside one graph, asynchronously; the
    device outputs equal the host ones."""
    import torch
    W, L, p, seed, n = 20, 300, 0.19, 11, 96
    h = pc.pc_inspect(W, L, p, seed, 0, n, mode=pc.PC_MODE_STREAM, bits_only=True)
    d = pc.pc_inspect(W, L, p, seed, 0, n, mode=pc.PC_MODE_STREAM, bits_only=True, device=True)
    torch.cuda.synchronize()
    d = {k: v.cpu().numpy() for k, v in d.items()}
    _check(d, h, "device outputs")
    assert int(d["n_percolating"][0]) == h["n_percolating"]


def test_blocked_host_loop_equals_graph(monkeypatch):
    """The host-driven passes (for profilers) give the graph's results."""
    W, L, p, seed, n = 32, 400, 0.17, 12, 24
    g = pc.pc_inspect(W, L, p, seed, 0, n, mode=pc.PC_MODE_STREAM, bits_only=True)
    monkeypatch.setenv("PC_STREAM_HOST_LOOP", "1")
    h = pc.pc_inspect(W, L, p, seed, 0, n, mode=pc.PC_MODE_STREAM, bits_only=True)
    _check(h, g, "host loop")
