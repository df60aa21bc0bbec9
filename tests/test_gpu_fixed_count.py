"""Fixed-count sample space (Sec. II.A: a random permutation of the N sites
puts exactly Np of them metallic) on the GPU: the occupancy bits against the
oracle's plain definition (the Np smallest keys (word, site index)) bit for
bit, and inspections of those configurations against the oracle."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
import paper_1401_2130_gb300 as pc

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


@pytest.mark.parametrize("W,L,frac,seed,cfg0,n", [
    (4, 16, 0.15, 1, 0, 64),      # tiny
    (8, 64, 0.2, 2, 1000, 16),    # p-sweep lattice
    (3, 7, 0.5, 9, 3, 33),        # N = 259: ragged last word
    (2, 5, 0.0, 5, 0, 4),         # no metallic site
    (2, 5, 1.0, 5, 0, 4),         # every site metallic
    (0, 1, 1.0, 7, 0, 3),         # one site
    (16, 64, 0.17, 4, 7, 6),      # N = 52,288
])
def test_fixed_count_bits_match_oracle(W, L, frac, seed, cfg0, n):
    import torch
    _, N = oracle.lattice_info(W, L)
    Np = int(round(frac * N))
    bits = pc.pc_occupancy_fixed(W, L, Np, seed, cfg0, n)
    torch.cuda.synchronize()
    got = bits.cpu().numpy().view(np.uint32)
    ref = oracle.pack_bits(oracle.occupancy_fixed(W, L, Np, seed, cfg0, n))
    assert np.array_equal(got, ref)


def test_fixed_count_equals_bernoulli_at_its_count():
    import torch
    W, L, p, seed = 6, 30, 0.2, 3
    bern = pc.pc_occupancy(W, L, p, seed, 0, 8)
    torch.cuda.synchronize()
    bern = bern.cpu().numpy().view(np.uint32)
    _, N = oracle.lattice_info(W, L)
    for c in range(8):
        Np = int(np.unpackbits(bern[c].view(np.uint8)).sum())
        f = pc.pc_occupancy_fixed(W, L, Np, seed, c, 1)
        torch.cuda.synchronize()
        assert np.array_equal(f.cpu().numpy().view(np.uint32)[0], bern[c])


def test_fixed_count_inspection_matches_oracle():
    import torch
    W, L, seed, n = 5, 40, 12, 200
    _, N = oracle.lattice_info(W, L)
    Np = int(round(0.25 * N))
    bits = pc.pc_occupancy_fixed(W, L, Np, seed, 0, n)
    g = pc.pc_inspect_occupancy(W, L, bits)
    occ = oracle.occupancy_fixed(W, L, Np, seed, 0, n)
    ref = oracle.inspect(W, L, occ=occ, mode="markov", threads=THREADS)
    assert np.array_equal(np.asarray(g["verdict"]).astype(np.int32), ref["verdict"])
    assert np.array_equal(g["first_hit"], ref["first_hit"])
    assert np.array_equal(g["m_stop"], ref["m_stop"])
    assert np.abs(np.asarray(g["mass"], np.float64) - ref["mass"]).max() <= 1e-5


def test_fixed_count_rejects_bad_counts():
    _, N = oracle.lattice_info(2, 5)
    for bad in (-1, N + 1):
        with pytest.raises(pc.PercolError) as e:
            pc.pc_occupancy_fixed(2, 5, bad, 1, 0, 1)
        assert e.value.status == pc.PC_ERR_ARG
