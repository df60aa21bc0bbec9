"""The lazy walk of the self-loop remark (Sec. II.B) through the C ABI:
pc_lazy_mass on the GPU inspection's outputs against the oracle's explicit
lazy chain hold * I + (1 - hold) * P in FP64 (mass within 1e-5 absolute,
and 1e-5 relative where the mass is not negligible)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1401_2130_gb300 as pc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("hold", [0.0, 0.25, 0.5, 0.9])
def test_lazy_mass_equals_oracle_lazy_chain(hold):
    W, L, p, seed, n = 2, 5, 0.55, 21, 40
    g = pc.pc_inspect(W, L, p, seed, 0, n)
    lazy = pc.pc_lazy_mass(g["first_hit"], g["mass"], hold)
    occ = oracle.occupancy(W, L, p, seed, 0, n)
    for c in range(n):
        a = oracle.first_passage_lazy(W, L, occ[c], 25, hold)
        fh = int(g["first_hit"][c])
        if fh > 0:
            assert np.all(a[: fh - 1] == 0.0) and a[fh - 1] > 0   # first hit unchanged
            assert abs(lazy[c] - a[fh - 1]) <= 1e-5
            assert lazy[c] == pytest.approx(a[fh - 1], rel=1e-5)
        else:
            assert not np.any(a) and lazy[c] == 0.0


def test_lazy_mass_device_buffers_and_aliasing():
    import torch
    # short fibres keep the first-passage masses far from FP32 underflow
    W, L, p, seed, n = 4, 4, 0.5, 21, 256
    host = pc.pc_inspect(W, L, p, seed, 0, n)
    want = pc.pc_lazy_mass(host["first_hit"], host["mass"], 0.3)
    d = pc.pc_inspect(W, L, p, seed, 0, n, device=True)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        got = pc.pc_lazy_mass(d["first_hit"], d["mass"], 0.3, stream=s)
        pc.pc_lazy_mass(d["first_hit"], d["mass"], 0.3, out=d["mass"], stream=s)  # in place
    s.synchronize()
    assert np.array_equal(got.cpu().numpy(), want)
    assert np.array_equal(d["mass"].cpu().numpy(), want)
    # the factor (0.7)^first_hit is applied to every percolating mass
    perc = host["verdict"] != 0
    assert perc.sum() > 50 and np.all(host["mass"][perc] > 1e-6)
    ratio = want[perc].astype(np.float64) / host["mass"][perc]
    assert np.allclose(ratio, 0.7 ** host["first_hit"][perc].astype(np.float64), rtol=1e-6)
