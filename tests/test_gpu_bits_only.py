"""PC_BITS_ONLY: the exact reached-set propagation alone (Sec. II.B -- only
whether the detector probability is zero decides percolation).  Verdicts,
first_hit and m_stop must equal the oracle's bit for bit (BFS and Markov
modes), in both solvers and in batches; mass is written 0."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
import paper_1401_2130_gb300 as pc

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


def _check(g, ref, what):
    assert np.array_equal(np.asarray(g["verdict"]).astype(np.int32), ref["verdict"]), what
    assert np.array_equal(np.asarray(g["first_hit"]), ref["first_hit"]), what
    assert np.array_equal(np.asarray(g["m_stop"]), ref["m_stop"]), what
    assert not np.any(np.asarray(g["mass"])), what


@pytest.mark.parametrize("W,L,p,seed,cfg0,n,mode", [
    (4, 16, 0.15, 1, 0, 1000, 0),                    # tiny, resident
    (8, 64, 0.19, 2, 0, 2000, 0),                    # p-sweep lattice near its threshold
    (8, 64, 0.3, 2, 0, 500, pc.PC_MODE_STREAM),      # the same lattice, streamed
    (16, 128, 0.2, 7, 5, 300, 0),                    # beyond shared memory: streamed
    (3, 1, 0.5, 3, 0, 64, 0),                        # L = 1
    (0, 40, 0.97, 4, 0, 256, 0),                     # single tube
    (5, 37, 0.0, 1, 0, 16, pc.PC_MODE_STREAM),       # nothing metallic
])
def test_bits_only_equals_oracle(W, L, p, seed, cfg0, n, mode):
    g = pc.pc_inspect(W, L, p, seed, cfg0, n, mode=mode, bits_only=True)
    ref = oracle.inspect(W, L, p=p, seed=seed, cfg0=cfg0, n=n, mode="bfs", threads=THREADS)
    _check(g, ref, (W, L, p, mode))
    assert g["n_percolating"] == int(ref["verdict"].sum())
    full = pc.pc_inspect(W, L, p, seed, cfg0, n, mode=mode)
    for k in ("verdict", "first_hit", "m_stop"):
        assert np.array_equal(full[k], g[k]), k


@pytest.mark.parametrize("mode", [pc.PC_MODE_RESIDENT, pc.PC_MODE_STREAM])
def test_bits_only_skips_the_fp_recursion(mode):
    # short fibres: the full inspection's first-passage masses are far from
    # FP32 underflow, so a zero mass shows that the recursion did not run
    W, L, p, seed, n = 4, 4, 0.5, 21, 256
    full = pc.pc_inspect(W, L, p, seed, 0, n, mode=mode)
    bits = pc.pc_inspect(W, L, p, seed, 0, n, mode=mode, bits_only=True)
    perc = full["verdict"] != 0
    assert perc.sum() > 50 and np.all(full["mass"][perc] > 1e-6)
    assert not np.any(bits["mass"])
    for k in ("verdict", "first_hit", "m_stop"):
        assert np.array_equal(full[k], bits[k]), k


def test_bits_only_markov_sample():
    # the Markov (FP64 CSR) oracle decides with the support of the iterate
    W, L, p, seed, n = 6, 24, 0.21, 11, 200
    g = pc.pc_inspect(W, L, p, seed, 0, n, bits_only=True)
    ref = oracle.inspect(W, L, p=p, seed=seed, n=n, mode="markov", threads=THREADS)
    _check(g, ref, "markov")


def test_bits_only_batch():
    specs = [(4, 8, 0.2, 3, 0, 400), (8, 64, 0.18, 3, 100, 300), (12, 200, 0.17, 3, 0, 64),
             (2, 500, 0.4, 3, 7, 32)]
    outs, res = pc.pc_batch_run(specs, bits_only=True)
    for sp, o, r in zip(specs, outs, res):
        W, L, p, seed, b, n = sp
        ref = oracle.inspect(W, L, p=p, seed=seed, cfg0=b, n=n, mode="bfs", threads=THREADS)
        _check(o, ref, sp)
        assert r["n_percolating"] == int(ref["verdict"].sum())
