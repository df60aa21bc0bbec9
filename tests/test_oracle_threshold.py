"""The oracle's critical word per configuration, and through it a pin of the
oracle's lattice (neighbour set and W, L) to the constants the paper prints.

With coupled draws a configuration percolates at p exactly when T(p) exceeds
its critical word w* (Sec. II.B: a path of metallic sites joins the two
ends).  w* is pinned by brute force (BFS verdicts at several p) and by closed
forms (a single column, a single layer).  Its empirical distribution is Pi(p)
of Eq. (5) at every p, which makes the finite-size-scaling analysis of
Sec. III (Eqs. (5), (7), (8)) cheap enough for the CPU suite: it must land
near p_c_inf = 0.1533 +- 0.0013 and alpha = -1.23.  A plausible misreading of
the neighbour set (the rod-contact table, in which each tube touches two
tubes of every adjacent column and none two rows away) is planted in the
oracle's adjacency and must fall outside that window."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle

THREADS = os.cpu_count() or 1


@pytest.mark.parametrize("W,L,seed,cfg0,n", [
    (4, 16, 3, 0, 300),
    (2, 40, 5, 17, 200),
    (6, 9, 11, 0, 150),
    (1, 2, 1, 0, 400),
])
def test_critical_word_decides_every_p(W, L, seed, cfg0, n):
    ws = oracle.critical_words(W, L, seed, cfg0, n, threads=THREADS)
    for p in (0.05, 0.15, 0.2, 0.25, 0.3, 0.4, 0.6, 1.0):
        v = oracle.inspect(W, L, p=p, seed=seed, cfg0=cfg0, n=n, mode="bfs", threads=THREADS)["verdict"]
        assert np.array_equal(v.astype(bool), ws < oracle.threshold(p)), p


def test_single_column_needs_every_tube():
    # W = 0: the column percolates only if all L tubes are metallic
    L, n = 12, 64
    ws = oracle.critical_words(0, L, 9, 0, n)
    words = oracle.site_words(0, L, 9, 0, n)
    assert np.array_equal(ws, words.max(axis=1).astype(np.uint64))


def test_single_layer_needs_one_site():
    # L = 1: start face = end face, so the smallest word decides (reading G12)
    W, n = 5, 64
    ws = oracle.critical_words(W, 1, 4, 0, n)
    words = oracle.site_words(W, 1, 4, 0, n)
    assert np.array_equal(ws, words.min(axis=1).astype(np.uint64))


def test_explicit_adjacency_is_the_lattice_default():
    W, L, n = 3, 10, 50
    a = oracle.critical_words(W, L, 2, 0, n)
    b = oracle.critical_words(W, L, 2, 0, n, adjacency=oracle.adjacency(W, L))
    assert np.array_equal(a, b)


_UP = ((1, 0), (-1, 1), (0, -1))
_DOWN = ((-1, 0), (1, -1), (0, 1))


def _rod_contact_adjacency(W, L):
    """The alternative reading of the 14 contacts: each of the 6 adjacent
    columns touched at two heights (one layer up and two down on the 'up'
    side, the mirror on the 'down' side), plus the two end contacts; no
    contacts two rows away.  Also 14 per site."""
    q, r, s = oracle.columns(W)
    A = q.size
    at = {(int(q[a]), int(r[a])): a for a in range(A)}
    nbr = np.full((A * L, 14), -1, np.int64)
    cnt = np.zeros(A * L, np.int32)
    for a in range(A):
        sg = int(s[a])
        offs = [(0, 0, 1), (0, 0, -1)]
        for dq, dr in _UP:
            offs += [(dq, dr, int(sg == 2)), (dq, dr, -int(sg != 2))]
        for dq, dr in _DOWN:
            offs += [(dq, dr, -int(sg == 0)), (dq, dr, int(sg != 0))]
        for t in range(L):
            i, k = t * A + a, 0
            for dq, dr, dt in offs:
                b = at.get((int(q[a]) + dq, int(r[a]) + dr))
                if b is not None and 0 <= t + dt < L:
                    nbr[i, k] = (t + dt) * A + b
                    k += 1
            cnt[i] = k
    return nbr, cnt


def _fss(adjacency_of, seed=6, n=1024):
    """Eq. (5) fitted to each size (the logistic distribution of w*/2^32 is
    Eq. (5) as a distribution function), then Eqs. (7) and (8)."""
    stats = pytest.importorskip("scipy.stats")
    from paper_1401_2130_gb300 import fss

    Ws, Ls, pcs, errs = [], [], [], []
    for W in (8, 12, 16):
        for ratio in (2, 1, 0.5, 0.25, 0.125):
            L = int(round(W / ratio))
            x = oracle.critical_words(W, L, seed, 0, n, adjacency=adjacency_of(W, L),
                                      threads=THREADS).astype(float) / 2.0**32
            loc, scale = stats.logistic.fit(x)
            Ws.append(W); Ls.append(L); pcs.append(loc); errs.append(np.sqrt(3.0 / n) * scale)
    f = fss.fit_fss(Ws, Ls, pcs, errs)
    r = sorted(f.slopes)
    (C0, C1, alpha), _ = fss.fit_slope_law(r, [f.slopes[k][0] for k in r], [f.slopes[k][1] for k in r])
    return f, alpha


def test_lattice_reproduces_paper_threshold():
    # Sec. III: p_c_inf = 0.1533 +- 0.0013 and alpha = -1.23.  Widths 8..16
    # carry a finite-size systematic of a few 1e-3 (at widths up to 32 the
    # same analysis gives 0.1558); the window is the one the GPU scan uses.
    f, alpha = _fss(lambda W, L: None)
    assert 0.150 < f.p_inf < 0.162, f.p_inf
    assert -1.30 < alpha < -1.17, alpha
    assert f.chi2 / f.dof < 4.0, (f.chi2, f.dof)


def test_rod_contact_reading_misses_paper_threshold():
    # the planted misreading percolates later: p_c_inf near 0.177
    f, _ = _fss(_rod_contact_adjacency)
    assert not 0.150 < f.p_inf < 0.162, f.p_inf
