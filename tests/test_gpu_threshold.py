"""GPU verdicts at many values of p against one oracle pass: a configuration
percolates at p exactly when T(p) exceeds its critical word (Sec. II.B, with
the coupled draws of the occupancy stream), so every p of a sweep is checked
against the same oracle output, in both solvers and in a batch."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
import paper_1401_2130_gb300 as pc

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


@pytest.mark.parametrize("W,L,seed,cfg0,n,mode", [
    (8, 64, 2, 0, 1000, 0),                     # the p-sweep lattice, resident
    (8, 64, 2, 3000, 200, pc.PC_MODE_STREAM),   # the same lattice, streamed
    (20, 160, 9, 0, 48, 0),                     # beyond shared memory
])
def test_verdicts_follow_critical_words(W, L, seed, cfg0, n, mode):
    ws = oracle.critical_words(W, L, seed, cfg0, n, threads=THREADS)
    for p in (0.12, 0.16, 0.18, 0.2, 0.22, 0.26, 0.35):
        g = pc.pc_inspect(W, L, p, seed, cfg0, n, mode=mode, bits_only=True)
        want = ws < oracle.threshold(p)
        assert np.array_equal(np.asarray(g["verdict"]).astype(bool), want), p
        assert g["n_percolating"] == int(want.sum())


def test_batch_sweep_follows_critical_words():
    W, L, seed, n = 12, 96, 4, 256
    ps = [0.15, 0.17, 0.18, 0.19, 0.2, 0.21, 0.23]
    ws = oracle.critical_words(W, L, seed, 0, n, threads=THREADS)
    outs, res = pc.pc_batch_run([(W, L, p, seed, 0, n) for p in ps])
    for p, o, r in zip(ps, outs, res):
        want = ws < oracle.threshold(p)
        assert np.array_equal(np.asarray(o["verdict"]).astype(bool), want), p
        assert r["n_percolating"] == int(want.sum())
