"""Finite-size-scaling analysis (Sec. III, Eqs. (5)-(9)) on synthetic data
with known parameters, and Eq. (9) against the number the paper prints."""
import os

import numpy as np
import pytest

pytest.importorskip("scipy")

from paper_1401_2130_gb300 import fss


def test_fermi_dirac_shape():
    # Eq. (5): 1/2 at p = p_c, 0 and 1 far below and above
    assert fss.fermi_dirac(0.2, 0.2, 0.01) == pytest.approx(0.5)
    assert fss.fermi_dirac(0.0, 0.2, 0.01) < 1e-8
    assert fss.fermi_dirac(1.0, 0.2, 0.01) > 1 - 1e-8
    # symmetric about p_c
    assert fss.fermi_dirac(0.23, 0.2, 0.01) == pytest.approx(1 - fss.fermi_dirac(0.17, 0.2, 0.01))


def test_fit_recovers_exact_curve():
    p = np.linspace(0.10, 0.30, 41)
    n = np.full(p.size, 10**7)
    k = np.round(n * fss.fermi_dirac(p, 0.1733, 0.0121))
    f = fss.fit_fermi_dirac(p, k, n)
    assert f.p_c == pytest.approx(0.1733, abs=2e-5)
    assert f.T == pytest.approx(0.0121, rel=2e-3)


def test_fit_on_binomial_samples_is_consistent():
    rng = np.random.default_rng(7)
    p = np.linspace(0.12, 0.26, 29)
    n = np.full(p.size, 1024)
    hits = 0
    for _ in range(40):
        k = rng.binomial(n, fss.fermi_dirac(p, 0.19, 0.015))
        f = fss.fit_fermi_dirac(p, k, n)
        hits += abs(f.p_c - 0.19) < 2 * f.p_c_err
    assert hits >= 32  # ~95% coverage of a 2-sigma interval


def test_fss_recovers_common_intercept_and_slopes():
    nu = fss.NU_3D
    W, L, pc, err = [], [], [], []
    for r, C in ((1.0, 0.05), (0.25, 0.8), (1 / 16, 6.0)):
        for Wv in (4, 8, 16, 32):
            Lv = Wv / r
            W.append(Wv); L.append(Lv); pc.append(0.1533 + C * Lv ** (-1 / nu)); err.append(1e-4)
    f = fss.fit_fss(W, L, pc, err)
    assert f.p_inf == pytest.approx(0.1533, abs=1e-9)
    for r, C in ((1.0, 0.05), (0.25, 0.8), (1 / 16, 6.0)):
        assert f.slopes[round(r, 12)][0] == pytest.approx(C, rel=1e-7)
    assert f.chi2 == pytest.approx(0.0, abs=1e-12)


def test_slope_law_fit():
    r = np.array([1.0, 0.5, 0.25, 0.125, 1 / 16, 1 / 32, 1 / 64])
    C = fss.slope_law(r, -0.83, 0.31, -1.23)
    (C0, C1, a), _ = fss.fit_slope_law(r, C)
    assert (C0, C1, a) == pytest.approx((-0.83, 0.31, -1.23), rel=1e-6)


def test_eq9_macroscopic_increment_matches_paper():
    # Sec. III: W = 10^6 and W/L = 10^-3 give an increment of 9.2e-8 over
    # p_c_inf with C0 = -0.83, C1 = 0.31, alpha = -1.23 (rounded constants
    # reproduce 9.0e-8)
    inc = fss.p_c_eq9(1e6, 1e9, 0.0, -0.83, 0.31, -1.23)
    assert 8.8e-8 < inc < 9.4e-8
    # Eq. (9) is Eq. (7) with Eq. (8) substituted
    W, L = 37.0, 600.0
    lhs = fss.p_c_eq9(W, L, 0.15, -0.83, 0.31, -1.23)
    rhs = 0.15 + fss.slope_law(W / L, -0.83, 0.31, -1.23) * L ** (-1 / fss.NU_3D)
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_decay_rate_recovers_exponential():
    L = np.array([4, 8, 16, 32, 64, 128, 256])
    n = np.full(L.size, 10**8)
    k = np.round(n * 0.97 * np.exp(-0.0123 * L))
    f = fss.decay_rate(L, k, n)
    assert f.lam == pytest.approx(0.0123, rel=1e-4)
    # fully percolating over the range: no decay
    assert fss.decay_rate(L, n, n).lam == 0.0


# ---------------------------------------------------------------------------
# The scan and length-scan orchestration, with the oracle's counts in place of
# the GPU batch (the GPU verdicts equal the oracle's bit for bit): a
# configuration percolates at p exactly when T(p) exceeds its critical word.
# ---------------------------------------------------------------------------

def _oracle_counts(monkeypatch):
    import oracle
    threads = os.cpu_count() or 1
    words = {}
    seen = []

    def measure(specs):
        out = []
        for (W, L, p, seed, b, n) in specs:
            seen.append((W, L, p, seed, b, n))
            have = words.get((W, L, seed), np.zeros(0, np.uint64))
            if have.size < b + n:
                extra = oracle.critical_words(W, L, seed, have.size, b + n - have.size, threads=threads)
                have = words[(W, L, seed)] = np.concatenate([have, extra])
            out.append(int((have[b:b + n] < oracle.threshold(p)).sum()))
        return out

    monkeypatch.setattr(fss, "measure", measure)
    return words, seen


def test_scan_fine_points_use_disjoint_configurations(monkeypatch):
    _, seen = _oracle_counts(monkeypatch)
    fss.scan([(4, 8), (6, 6)], seed=3, n_coarse=64, n_fine=128, fine_points=7)
    for size in ((4, 8), (6, 6)):
        fine = [s for s in seen if s[:2] == size and s[5] == 128]
        assert len(fine) == 7
        starts = sorted(s[4] for s in fine)
        assert starts == [j * 128 for j in range(7)]


def test_scan_and_extrapolation_on_oracle_counts(monkeypatch):
    # Sec. III on the oracle's lattice through the same code the GPU scan
    # uses: each size's Eq. (5) fit agrees with the logistic fit of all its
    # configurations' critical words within the fit's own (independent-count)
    # errors, and Eqs. (7)-(8) land in the paper's window
    stats = pytest.importorskip("scipy.stats")
    words, _ = _oracle_counts(monkeypatch)
    sizes = [(W, int(round(W / r))) for W in (8, 12, 16) for r in (2, 1, 0.5, 0.25, 0.125)]
    curves = fss.scan(sizes, seed=6, n_coarse=256, n_fine=256)
    pulls = []
    for (W, L), (f, p, k, n) in curves.items():
        x = words[(W, L, 6)][: 13 * 256].astype(float) / 2.0**32
        loc, scale = stats.logistic.fit(x)
        pulls.append((f.p_c - loc) / f.p_c_err)
    pulls = np.asarray(pulls)
    assert np.sqrt(np.mean(pulls ** 2)) < 2.0, pulls
    fit, law = fss.extrapolate(curves)
    assert 0.150 < fit.p_inf < 0.162, fit
    assert -1.30 < law[0][2] < -1.17, law


def test_length_statements_on_oracle_counts(monkeypatch):
    # Sec. III / Fig. 6(a) on the oracle's lattice (reading G13): at p = 0.3 a
    # W = 6 fibre keeps percolating over W/L >= 1/16, while a W = 3 fibre
    # loses percolation exponentially with its length, more than ten times
    # faster
    _oracle_counts(monkeypatch)
    six = fss.length_scan(6, [6, 24, 96], [0.3], 1024, 8)[0.3]
    assert np.all(six[1] / six[2] >= 0.99), six[1]
    three = fss.length_scan(3, [3, 6, 12, 24, 48, 96], [0.3], 1024, 8)[0.3]
    assert np.all(np.diff(three[1]) <= 0), three[1]
    assert three[3].lam > 10 * max(six[3].lam, 1e-6), (three[3], six[3])
