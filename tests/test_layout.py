"""The padded-row plane layout and the strip gathers of the tiled FP sweep,
checked on the host: every side-contact read of every valid output lands on
the right neighbour column, or on a zero entry when the neighbour lies
outside the hexagon; every read of every strip stays within its own plane
(so one contiguous segment per plane feeds a chunk of strips).  The run formulas below are the ones the kernels use."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1401_2130_gb300 as pc
from paper_1401_2130_gb300 import _build

# (run, start offset relative to 3s (plus the row offset), rows delta)
RUNS = {"U": (-2, +1), "D": (-1, -1), "C": (-1, 0), "E": (-1, +2), "F": (+1, -2)}
ROW_K = {-2: 0, -1: 1, +1: 2, +2: 3}
# direction -> (dq, dr, run, index offset: run index = j + k)
DIRS = {0: (1, 1, "U", 3), 4: (-2, 1, "U", 0), 7: (-1, 1, "U", 1), 11: (0, 1, "U", 2),
        3: (-1, -1, "D", 0), 1: (2, -1, "D", 3), 8: (0, -1, "D", 1), 10: (1, -1, "D", 2),
        6: (1, 0, "C", 2), 9: (-1, 0, "C", 0), 5: (-1, 2, "E", 0), 2: (1, -2, "F", 0)}


@pytest.fixture(scope="module", autouse=True)
def lib():
    _build.build()
    pc.load()


@pytest.mark.parametrize("W", [0, 1, 2, 3, 4, 7, 8, 16, 33, 64])
def test_strip_gathers_hit_the_right_neighbours(W):
    lay = pc.pc_lattice_layout(W)
    P, ppos, pcol = lay["P"], lay["ppos"], lay["pcol"]
    q, r, s = oracle.columns(W)
    A = len(q)
    assert np.array_equal(pcol[ppos], np.arange(A))
    assert (pcol >= 0).sum() == A
    assert P % 4 == 0
    # sublattice = position mod 3 for every column
    assert np.all(ppos % 3 == (q - r) % 3)
    idx = {(int(q[a]), int(r[a])): a for a in range(A)}

    def value_at(pos):
        """column at a plane position: every read stays inside its own plane."""
        assert 0 <= pos < P, pos
        return pcol[pos]

    for k in range(lay["n_strips"]):
        st = lay["s_begin"] + k
        ri = int(lay["strip_row"][k])
        b = 3 * st
        row = ri - W
        off = {0: 0, **{d: int(lay["row_off"][ri, ROW_K[d]]) for d in (-2, -1, 1, 2)}}
        starts = {name: b + c + off[dr] for name, (c, dr) in RUNS.items()}
        lens = {"U": 6, "D": 6, "C": 5, "E": 3, "F": 3}
        for name in starts:  # every read of every strip stays near its plane
            for i in range(lens[name]):
                value_at(starts[name] + i)
        for j in range(3):
            a = pcol[b + j] if 0 <= b + j < P else -1
            if a < 0:
                continue
            assert r[a] == row and (q[a] - r[a]) % 3 == j
            for d, (dq, dr, name, kk) in DIRS.items():
                got = value_at(starts[name] + j + kk)
                want = idx.get((int(q[a]) + dq, int(r[a]) + dr), -1)
                assert got == want, (W, st, j, d, got, want)


def test_static_entry_point_tables_cover_its_widest_lattice():
    # pc_inspect_static keeps the layout of every accepted width (W <= 51) in
    # fixed tables of 9216 plane entries and 9216 / 3 + 2 strips
    for W in range(0, 52):
        lay = pc.pc_lattice_layout(W)
        assert lay["P"] <= 9216, (W, lay["P"])
        assert lay["n_strips"] <= 9216 // 3 + 2, (W, lay["n_strips"])
