"""Serving loop (pc_server_*): continuous batching.  Queries submitted while
others run are admitted as memory and slots free up; every query's result in
the mix equals its result alone (pc_inspect) and the oracle's."""
from __future__ import annotations

import os
import time

import numpy as np
import pytest

import oracle
import paper_1401_2130_gb300 as pc

pytestmark = pytest.mark.gpu

MASS_TOL = 1e-5
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    pc.build()
    pc.load()
    torch.cuda.init()


def _same(a, b, what):
    for k in ("verdict", "first_hit", "m_stop"):
        assert np.array_equal(np.asarray(a[k]).astype(np.int64), np.asarray(b[k]).astype(np.int64)), (what, k)
    err = np.abs(np.asarray(a["mass"], np.float64) - np.asarray(b["mass"], np.float64))
    assert err.max(initial=0.0) <= MASS_TOL, (what, err.max())


def _mix(seed=0, n=24):
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n):
        W = int(rng.integers(2, 20))
        L = int(round(W * np.exp(rng.uniform(0, np.log(12)))))
        p = float(rng.uniform(0.14, 0.3))
        specs.append((W, max(L, 1), p, 100 + i, int(rng.integers(0, 1000)), int(rng.integers(20, 300))))
    return specs


def test_results_in_the_mix_equal_alone_and_oracle():
    specs = _mix()
    srv = pc.Server(hbm_budget_bytes=2 << 30, max_slots=48, max_slots_per_query=16, ticks_per_poll=4)
    try:
        tickets = [srv.submit(sp) for sp in specs]
        got = {}
        deadline = time.time() + 120
        while len(got) < len(tickets) and time.time() < deadline:
            for t in tickets:
                if t not in got:
                    r = srv.poll(t, timeout_s=0.01)
                    if r is not None:
                        got[t] = r
        assert len(got) == len(tickets)
        st = srv.stats()
        assert st["completed"] == len(specs) and st["p99_ms"] >= st["p50_ms"] > 0
    finally:
        srv.close()
    kinds = {got[t]["solver"] for t in tickets}
    assert kinds == {"resident", "streamed"}
    for sp, t in zip(specs, tickets):
        W, L, p, seed, b, n = sp
        alone = pc.pc_inspect(W, L, p, seed, b, n)
        _same(got[t], alone, sp)
        assert got[t]["n_percolating"] == alone["n_percolating"]
    for sp, t in list(zip(specs, tickets))[:8]:
        W, L, p, seed, b, n = sp
        ref = oracle.inspect(W, L, p=p, seed=seed, cfg0=b, n=n, mode="markov", threads=THREADS)
        _same(got[t], ref, sp)


def test_arrivals_while_running_and_footprint_admission():
    """A small arena: later queries wait for memory, then run; results exact."""
    specs = [(16, 160, 0.2, 7, 0, 60), (20, 100, 0.2, 8, 0, 60), (6, 30, 0.25, 9, 0, 400),
             (18, 120, 0.19, 10, 0, 50)]
    srv = pc.Server(hbm_budget_bytes=16 << 20, max_slots=16, max_slots_per_query=8, ticks_per_poll=2)
    try:
        tickets = []
        for sp in specs:
            tickets.append(srv.submit(sp))
            time.sleep(0.01)  # arrive while earlier ones run
        res = {t: None for t in tickets}
        deadline = time.time() + 120
        while any(v is None for v in res.values()) and time.time() < deadline:
            for t in tickets:
                if res[t] is None:
                    res[t] = srv.poll(t, timeout_s=0.01)
    finally:
        srv.close()
    for sp, t in zip(specs, tickets):
        W, L, p, seed, b, n = sp
        assert res[t] is not None, sp
        _same(res[t], pc.pc_inspect(W, L, p, seed, b, n), sp)


def test_errors_busy_cancel_and_oversize():
    srv = pc.Server(hbm_budget_bytes=32 << 20, max_slots=4, max_slots_per_query=4, ticks_per_poll=1)
    try:
        # larger than the whole budget: rejected at submit
        with pytest.raises(pc.PercolError) as e:
            srv.submit((64, 4096, 0.2, 1, 0, 10))
        assert e.value.status == pc.PC_ERR_OOM
        big = srv.submit((12, 400, 0.3, 1, 0, 64))
        queued = [srv.submit((12, 400, 0.3, 2 + i, 0, 64)) for i in range(3)]
        assert srv.poll(big, timeout_s=0.0) is None  # still running: PC_ERR_BUSY
        srv.cancel(queued[-1])
        with pytest.raises(pc.PercolError) as e:
            srv.poll(queued[-1])
        assert e.value.status == pc.PC_ERR_CANCELLED
        r = srv.poll(big, timeout_s=120.0)
        assert r is not None
        with pytest.raises(pc.PercolError) as e:
            srv.poll(12345)
        assert e.value.status == pc.PC_ERR_ARG
    finally:
        srv.close()  # remaining queued tickets are cancelled


def test_max_width_bounds_streamed_queries():
    # the staging ring is sized for max_W: wider HBM-slot lattices are refused,
    # resident ones of any accepted width still run
    srv = pc.Server(hbm_budget_bytes=256 << 20, max_slots=8, max_slots_per_query=8, ticks_per_poll=2,
                    max_W=8)
    try:
        with pytest.raises(pc.PercolError) as e:
            srv.submit((12, 400, 0.3, 1, 0, 4))
        assert e.value.status == pc.PC_ERR_ARG
        specs = [(8, 300, 0.25, 3, 0, 16), (4, 16, 0.2, 3, 0, 40)]
        tickets = [srv.submit(sp) for sp in specs]
        for sp, t in zip(specs, tickets):
            r = srv.poll(t, timeout_s=120.0)
            assert r is not None
            _same(r, pc.pc_inspect(*sp), sp)
    finally:
        srv.close()
