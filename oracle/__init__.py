"""CPU oracle for the Markov-chain percolation inspection (arXiv:1401.2130).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The GPU library neither imports nor links it; the two share no code.

The arithmetic lives in ``percol_oracle.c`` (plain C, FP64, OpenMP over
configurations); this module compiles it with gcc and marshals numpy arrays.
Every function names the passage of the paper it follows:

* ``philox4x32_10``      -- Salmon et al., SC'11 (Philox-4x32, 10 rounds)
* ``lattice_info`` / ``columns`` / ``adjacency`` -- Sec. II.A, Fig. 1
* ``occupancy``          -- Sec. II.A (Bernoulli(p) per site)
* ``inspect``            -- Sec. II.B, Eqs. (1)-(4); modes 'markov' (explicit
  CSR P with detector, FP64 forward recursion), 'markov_full' (same, but run
  on to N_max after the reached set stops growing), 'bfs', 'unionfind'
* ``first_passage``      -- Appendix Eq. (A.3): forward and backward forms
* ``first_passage_dense``-- Eq. (3) on an explicit matrix (Fig. 2)
* ``first_passage_lazy`` -- the self-loop remark of Sec. II.B: the lazy chain
  hold * I + (1 - hold) * P
* ``site_words`` / ``occupancy_fixed`` -- Sec. II.A: the fixed-count sample
  space (the Np smallest keys (word, site))
* ``critical_words``     -- Sec. II.B spanning path with coupled draws: the
  word below which each configuration percolates, i.e. its verdict at every p
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "percol_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODES = {"markov": 0, "bfs": 1, "unionfind": 2, "markov_full": 3}
STAT_FIELDS = ("n0", "Np", "Nb", "dropped", "residual", "absorbed",
               "fp_first_nonzero", "nmax_ok")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-Wall",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i32, i64, u64, dbl, vp = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                      ctypes.c_double, ctypes.c_void_p)
            lib.oracle_philox4x32_10.argtypes = [vp, vp, vp]
            lib.oracle_philox4x32_10.restype = None
            lib.oracle_threshold.argtypes = [dbl]
            lib.oracle_threshold.restype = u64
            lib.oracle_lattice_info.argtypes = [i32, i32, vp, vp]
            lib.oracle_columns.argtypes = [i32, vp, vp, vp]
            lib.oracle_adjacency.argtypes = [i32, i32, vp, vp]
            lib.oracle_occupancy.argtypes = [i32, i32, dbl, u64, i64, i64, vp]
            lib.oracle_site_words.argtypes = [i32, i32, u64, i64, i64, vp]
            lib.oracle_inspect.argtypes = [i32, i32, vp, dbl, u64, i64, i64, i32, i32,
                                           vp, vp, vp, vp, vp]
            lib.oracle_first_passage.argtypes = [i32, i32, vp, ctypes.c_int32, vp, vp]
            lib.oracle_first_passage_dense.argtypes = [i32, vp, i32, i32, i32, vp]
            lib.oracle_max_threads.argtypes = []
            lib.oracle_critical_words.argtypes = [i32, i32, vp, vp, u64, i64, i64, i32, vp]
            lib.oracle_first_passage_lazy.argtypes = [i32, i32, vp, ctypes.c_int32, dbl, vp]
            for f in ("oracle_lattice_info", "oracle_columns", "oracle_adjacency",
                      "oracle_occupancy", "oracle_site_words", "oracle_inspect", "oracle_first_passage",
                      "oracle_first_passage_dense", "oracle_max_threads", "oracle_critical_words",
                      "oracle_first_passage_lazy"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _check(st: int, what: str):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: 4 x uint32 counter, 2 x uint32 key -> 4 x uint32."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    assert c.shape == (4,) and k.shape == (2,)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def threshold(p: float) -> int:
    """T = floor(p * 2^32): a site is metallic iff its 32-bit word is < T."""
    return int(_load().oracle_threshold(float(p)))


def lattice_info(W: int, L: int) -> tuple[int, int]:
    """(A, N): number of columns of the hexagon of radius W, and A * L sites."""
    a = np.zeros(1, np.int64)
    n = np.zeros(1, np.int64)
    _check(_load().oracle_lattice_info(W, L, _ptr(a), _ptr(n)), "lattice_info")
    return int(a[0]), int(n[0])


def columns(W: int):
    """Axial (q, r) and sublattice sigma of each column in canonical order."""
    A, _ = lattice_info(W, 1)
    q = np.zeros(A, np.int32); r = np.zeros(A, np.int32); s = np.zeros(A, np.int32)
    _check(_load().oracle_columns(W, _ptr(q), _ptr(r), _ptr(s)), "columns")
    return q, r, s


def adjacency(W: int, L: int):
    """Lattice adjacency [N][14] (-1 padded) and per-site neighbour count."""
    _, N = lattice_info(W, L)
    nbr = np.full((N, 14), -1, np.int64)
    cnt = np.zeros(N, np.int32)
    _check(_load().oracle_adjacency(W, L, _ptr(nbr), _ptr(cnt)), "adjacency")
    return nbr, cnt


def occupancy(W: int, L: int, p: float, seed: int, cfg0: int, n: int) -> np.ndarray:
    """Occupancy bytes [n][N] of configurations cfg0..cfg0+n-1."""
    _, N = lattice_info(W, L)
    occ = np.zeros((n, N), np.uint8)
    _check(_load().oracle_occupancy(W, L, float(p), int(seed) & (2**64 - 1), cfg0, n,
                                    _ptr(occ)), "occupancy")
    return occ


def site_words(W: int, L: int, seed: int, cfg0: int, n: int) -> np.ndarray:
    """The 32-bit random word of each site [n][N] (the Bernoulli draw's stream)."""
    _, N = lattice_info(W, L)
    w = np.zeros((n, N), np.uint32)
    _check(_load().oracle_site_words(W, L, int(seed) & (2**64 - 1), cfg0, n, _ptr(w)), "site_words")
    return w


def critical_words(W: int, L: int, seed: int, cfg0: int, n: int, adjacency=None,
                   threads: int = 0) -> np.ndarray:
    """Critical word w* of each configuration [n] (uint64): it percolates at p
    exactly when threshold(p) > w*, so Pi(p) for every p comes from one pass
    (Sec. II.B spanning path, union-find in increasing word order).
    ``adjacency`` = (nbr [N][14], count [N]) as ``adjacency`` returns it, to
    run another neighbour table; None = the lattice's own."""
    _, N = lattice_info(W, L)
    out = np.zeros(n, np.uint64)
    nbr = cnt = None
    if adjacency is not None:
        nbr = np.ascontiguousarray(adjacency[0], dtype=np.int64)
        cnt = np.ascontiguousarray(adjacency[1], dtype=np.int32)
        if nbr.shape != (N, 14) or cnt.shape != (N,) or np.any(cnt > 14) or np.any(cnt < 0):
            raise ValueError("adjacency must be ([N][14], [N]) with counts <= 14")
        if N and (nbr.max() >= N or any(np.any(nbr[i, :c] < 0) for i, c in enumerate(cnt) if c)):
            raise ValueError("adjacency entries out of range")
    _check(_load().oracle_critical_words(W, L, _ptr(nbr), _ptr(cnt), int(seed) & (2**64 - 1), cfg0, n,
                                          threads, _ptr(out)), "critical_words")
    return out


def occupancy_fixed(W: int, L: int, n_metallic: int, seed: int, cfg0: int, n: int) -> np.ndarray:
    """Fixed-count occupancy bytes [n][N] (Sec. II.A: a random permutation of
    the N sites puts exactly Np = n_metallic of them metallic).  The
    permutation sorts the sites by their random word, ties by site index; the
    first Np sites of it are metallic."""
    _, N = lattice_info(W, L)
    if not 0 <= n_metallic <= N:
        raise ValueError("n_metallic must be in [0, N]")
    words = site_words(W, L, seed, cfg0, n)
    occ = np.zeros((n, N), np.uint8)
    idx = np.arange(N)
    for c in range(n):
        order = np.lexsort((idx, words[c]))  # primary key: word, then index
        occ[c, order[:n_metallic]] = 1
    return occ


def pack_bits(occ: np.ndarray) -> np.ndarray:
    """Pack [n][N] bytes into [n][ceil(N/32)] uint32 words, bit (i & 31) of
    word (i >> 5) = site i."""
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    n, N = occ.shape
    words = (N + 31) // 32
    padded = np.zeros((n, words * 32), np.uint8)
    padded[:, :N] = occ
    bits = padded.reshape(n, words, 32).astype(np.uint64)
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    return (bits * weights).sum(axis=2).astype(np.uint32)


def unpack_bits(words: np.ndarray, N: int) -> np.ndarray:
    words = np.ascontiguousarray(words, dtype=np.uint32)
    n = words.shape[0]
    shifts = np.arange(32, dtype=np.uint32)
    bits = ((words[:, :, None] >> shifts) & 1).astype(np.uint8)
    return bits.reshape(n, -1)[:, :N]


def inspect(W: int, L: int, *, p: float = 0.0, seed: int = 0, cfg0: int = 0,
            n: int | None = None, occ: np.ndarray | None = None,
            mode: str = "markov", threads: int = 0, stats: bool = False) -> dict:
    """Inspect configurations (drawn from the stream, or explicit ``occ``).

    Returns numpy arrays: verdict (int32 0/1), first_hit (-1 if none),
    m_stop, mass (FP64, a_{first_hit}) and, with ``stats``, a dict of the
    per-configuration diagnostics of Markov mode.
    """
    _, N = lattice_info(W, L)
    if occ is not None:
        occ = np.ascontiguousarray(occ, dtype=np.uint8)
        if occ.ndim == 1:
            occ = occ[None, :]
        assert occ.shape[1] == N, (occ.shape, N)
        n = occ.shape[0]
    assert n is not None
    v = np.zeros(n, np.int32); fh = np.zeros(n, np.int32)
    ms = np.zeros(n, np.int32); mass = np.zeros(n, np.float64)
    st = np.zeros((n, 8), np.float64) if stats else None
    _check(_load().oracle_inspect(W, L, _ptr(occ), float(p), int(seed) & (2**64 - 1),
                                  cfg0, n, MODES[mode], threads, _ptr(v), _ptr(fh),
                                  _ptr(ms), _ptr(mass), _ptr(st)), "inspect")
    out = {"verdict": v, "first_hit": fh, "m_stop": ms, "mass": mass}
    if stats:
        out["stats"] = {k: st[:, i] for i, k in enumerate(STAT_FIELDS)}
    return out


def first_passage(W: int, L: int, occ: np.ndarray, mmax: int):
    """(forward a_m, backward mu_0^T f^(m)) for m = 1..mmax (Appendix)."""
    _, N = lattice_info(W, L)
    occ = np.ascontiguousarray(occ, dtype=np.uint8).reshape(N)
    fw = np.zeros(mmax, np.float64); bw = np.zeros(mmax, np.float64)
    _check(_load().oracle_first_passage(W, L, _ptr(occ), mmax, _ptr(fw), _ptr(bw)),
           "first_passage")
    return fw, bw


def first_passage_lazy(W: int, L: int, occ: np.ndarray, mmax: int, hold: float) -> np.ndarray:
    """Forward a_m, m = 1..mmax, of the lazy walk hold * I + (1 - hold) * P
    (the self-loop remark of Sec. II.B); hold in [0, 1)."""
    _, N = lattice_info(W, L)
    occ = np.ascontiguousarray(occ, dtype=np.uint8).reshape(N)
    fw = np.zeros(mmax, np.float64)
    _check(_load().oracle_first_passage_lazy(W, L, _ptr(occ), mmax, float(hold), _ptr(fw)),
           "first_passage_lazy")
    return fw


def first_passage_dense(P: np.ndarray, j0: int, i0: int, mmax: int) -> np.ndarray:
    """Eq. (3): P_{i0}[tau_{j0} = m], m = 1..mmax, for a dense matrix P."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    n = P.shape[0]
    out = np.zeros(mmax, np.float64)
    _check(_load().oracle_first_passage_dense(n, _ptr(P), j0, i0, mmax, _ptr(out)),
           "first_passage_dense")
    return out


def site_updates(A: int, L: int, verdict, first_hit, m_stop) -> int:
    """Site-updates the forward recursion performs: every step m that computes
    mu_m sweeps the causal window of min(m + 1, L) tube layers (A sites each).
    A percolating configuration computes mu_1..mu_{first_hit-1} (the last step
    only reads the detector); a non-percolating one mu_1..mu_{m_stop}."""
    verdict = np.asarray(verdict); first_hit = np.asarray(first_hit)
    m_stop = np.asarray(m_stop)
    M = np.where(verdict != 0, first_hit - 1, m_stop).astype(np.int64)
    M = np.maximum(M, 0)
    # sum_{m=1}^{M} min(m+1, L)
    k = np.minimum(M, L - 1)            # steps with window m+1 <= L
    s = k * (k + 3) // 2                # sum_{m=1}^{k} (m+1)
    s += np.maximum(M - k, 0) * L
    return int((s * A).sum())
