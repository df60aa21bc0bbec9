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


# strip-pair runs of the streamed solver: (name, start relative to 6h (plus
# the row offset), rows delta, 64-bit loads)
PAIR_RUNS = {"U": (-2, +1, 5), "D": (-2, -1, 5), "C": (-2, 0, 5), "E": (-2, +2, 4), "F": (0, -2, 4)}


@pytest.mark.parametrize("W", [0, 1, 2, 3, 4, 7, 8, 16, 33, 64, 100])
def test_strip_pair_layout_of_the_streamed_solver(W):
    """The paired layout: even row offsets (aligned 64-bit loads), no strip
    pair holding columns of two rows, every 64-bit read of every pair inside
    the plane, and every site of a pair reading its true neighbours through
    its strip's runs at the pair's row offsets."""
    lay = pc.pc_stream_layout(W)
    P, ppos, pcol = lay["P"], lay["ppos"], lay["pcol"]
    sb, ns = lay["s_begin"], lay["n_strips"]
    q, r, s = oracle.columns(W)
    A = len(q)
    assert P % 16 == 0
    assert np.array_equal(pcol[ppos], np.arange(A)) and (pcol >= 0).sum() == A
    assert np.all(ppos % 3 == (q - r) % 3)
    assert np.all(lay["row_off"] % 2 == 0)
    idx = {(int(q[a]), int(r[a])): a for a in range(A)}
    h_begin, h_end = sb // 2, (sb + ns + 1) // 2
    for h in range(h_begin, h_end):
        b = 6 * h
        rows = {int(r[a]) for a in pcol[b:b + 6] if a >= 0}
        assert len(rows) <= 1, (W, h, rows)
        st = min(max(2 * h + 1, sb), sb + ns - 1)
        ri = int(lay["strip_row"][st - sb])
        if rows:
            assert rows == {ri - W}, (W, h, rows, ri)
        off = {0: 0, **{d: int(lay["row_off"][ri, ROW_K[d]]) for d in (-2, -1, 1, 2)}}
        for name, (c, dr, nload) in PAIR_RUNS.items():
            start = b + c + off[dr]
            assert start % 2 == 0 and 0 <= start and start + 2 * nload <= P, (W, h, name)
        for j in range(6):  # every site of the pair, through its strip's runs
            a = pcol[b + j]
            if a < 0:
                continue
            bs = b + 3 * (j // 3)
            starts = {name: bs + cc + off[dr] for name, (cc, dr) in RUNS.items()}
            for d, (dq, dr, name, kk) in DIRS.items():
                got = pcol[starts[name] + j % 3 + kk]
                want = idx.get((int(q[a]) + dq, int(r[a]) + dr), -1)
                assert got == want, (W, h, j, d, got, want)


def test_static_entry_point_tables_cover_its_widest_lattice():
    # pc_inspect_static keeps the layout of every accepted width (W <= 51) in
    # fixed tables of 9216 plane entries and 9216 / 3 + 2 strips
    for W in range(0, 52):
        lay = pc.pc_lattice_layout(W)
        assert lay["P"] <= 9216, (W, lay["P"])
        assert lay["n_strips"] <= 9216 // 3 + 2, (W, lay["n_strips"])
