"""Seeded "wire" occupancies for mass parity at long first-passage times.

A wire is an induced path of metallic sites: every site of the path touches
only its predecessor and its successor (Sec. II.A contacts), and no other
site is metallic.  It starts at one site of the t = 0 layer and ends at its
only site of the t = L-1 layer.  On such a configuration the walk of
Sec. II.B has deg = 1 at the start, deg = 2 inside the wire and deg = 2 at the
end (one contact plus the detector edge), so the first hit is at
m = (number of wire sites) and the absorbed mass there is exactly
2^-(sites - 1): each step halves the frontier's probability.  Every partial
sum and product on the way is a power of two, so FP32 holds that value
exactly down to 2^-149, the smallest subnormal.

The path is built from the oracle's contact table (the neighbour set of
Sec. II.A derived from the FCC geometry), steered through random waypoints
across the hexagon so that it runs through many rows, columns and layers.
This module only builds inputs; it holds none of the method's arithmetic.
"""
from __future__ import annotations

import numpy as np

import oracle


def column_contacts(W: int):
    """(A, contacts): contacts[a] = list of (column b, tube shift dt) of the
    14 contacts of a site of column a, read from the oracle's adjacency of
    the middle layer of a 3-layer lattice."""
    A, _ = oracle.lattice_info(W, 3)
    nbr, cnt = oracle.adjacency(W, 3)
    contacts = []
    for a in range(A):
        i = A + a
        contacts.append([(int(j % A), int(j // A) - 1) for j in nbr[i, :cnt[i]]])
    return A, contacts


def _hex_dist(q0, r0, q1, r1):
    dq, dr = q1 - q0, r1 - r0
    return (abs(dq) + abs(dr) + abs(dq + dr)) // 2


def wire(W: int, L: int, rng: np.random.Generator, contacts, qr, max_sites: int = 150,
         n_waypoints: int = 2, spread: int | None = None, tries: int = 200):
    """One wire as a list of sites (t, a), or raises RuntimeError.

    qr = (q[A], r[A]) axial coordinates of the columns (oracle.columns);
    spread = largest hexagon distance of a waypoint from the previous one
    (None: anywhere in the hexagon)."""
    q, r = qr
    A = len(contacts)
    for _ in range(tries):
        a0 = int(rng.integers(A))
        wps, prev = [], a0
        for _ in range(n_waypoints):
            if spread is None:
                nxt = int(rng.integers(A))
            else:
                near = np.flatnonzero((np.abs(q - q[prev]) + np.abs(r - r[prev])
                                       + np.abs(q + r - q[prev] - r[prev])) // 2 <= spread)
                nxt = int(near[rng.integers(len(near))])
            wps.append(nxt)
            prev = nxt
        # tube targets of the waypoints rise toward the far end
        twps = sorted(int(rng.integers(1, max(2, L - 1))) for _ in range(n_waypoints))
        path = [(0, a0)]
        on = {(0, a0)}
        k = 0
        ok = L == 1
        while not ok and len(path) < max_sites:
            t, a = path[-1]
            final = k >= len(wps)
            tgt_a = path[-1][1] if final else wps[k]
            tgt_t = L - 1 if final else twps[k]
            best, best_s = None, None
            for b, dt in contacts[a]:
                s = (t + dt, b)
                if not 0 <= s[0] < L or s in on:
                    continue
                # the start layer holds only the first site, the end layer only the last
                if s[0] == 0 or (s[0] == L - 1 and not final):
                    continue
                # induced path: s touches no wire site other than the current one
                clash = False
                for c, dc in contacts[b]:
                    u = (s[0] + dc, c)
                    if u != (t, a) and u in on:
                        clash = True
                        break
                if clash:
                    continue
                score = (_hex_dist(q[b], r[b], q[tgt_a], r[tgt_a]) + abs(s[0] - tgt_t)
                         + 0.75 * rng.random())
                if best_s is None or score < best_s:
                    best, best_s = s, score
            if best is None:
                break
            path.append(best)
            on.add(best)
            if best[0] == L - 1:
                ok = True
                break
            if not final and best[1] == tgt_a and abs(best[0] - tgt_t) <= 1:
                k += 1
        if ok:
            return path
    raise RuntimeError(f"no wire found for W={W} L={L} within {max_sites} sites")


def wire_occupancies(W: int, L: int, n: int, seed: int, max_sites: int = 150,
                     n_waypoints: int = 2, spread: int | None = None):
    """n wire configurations [n][N] (uint8) and their site counts."""
    A, contacts = column_contacts(W)
    q, r, _ = oracle.columns(W)
    rng = np.random.default_rng(seed)
    occ = np.zeros((n, A * L), np.uint8)
    sites = np.zeros(n, np.int64)
    for c in range(n):
        path = wire(W, L, rng, contacts, (q, r), max_sites=max_sites, n_waypoints=n_waypoints,
                    spread=spread)
        for t, a in path:
            occ[c, t * A + a] = 1
        sites[c] = len(path)
    return occ, sites
