"""Finite-size scaling of the percolation probability (Sec. III, Eqs. (5)-(9)).

Host-side analysis of Pi(p) curves that the GPU inspection produces:

* Eq. (5): Pi(p) of one lattice size follows a Fermi-Dirac-shaped curve
  1 / (1 + exp((p_c - p) / T)); p_c is the size's effective threshold
  (Pi = 1/2) and T the width of the transition.  Fitted by binomial maximum
  likelihood on (p, percolating count, configurations).
* Eq. (7): p_c(W, L) = p_c_inf + C(W/L) * L^(-1/nu), nu = 0.88 in 3-D
  (Eq. (6)): sizes of one aspect ratio W/L lie on a line in L^(-1/nu), and all
  lines share the intercept p_c_inf.  Fitted jointly by weighted linear least
  squares (one intercept, one slope per aspect ratio).
* Eq. (8): C(W/L) = C0 + C1 (W/L)^alpha, fitted to the slopes.
* Eq. (9): p_c = p_c_inf + C0 L^(-1/nu) + C1 W^alpha L^(-alpha - 1/nu).

Nothing here touches the inspection itself; the inputs are the per-size
percolating counts that ``pc_inspect`` / ``pc_batch_run`` return.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

NU_3D = 0.88  # universal correlation-length exponent in 3-D (Eq. (6))


def fermi_dirac(p, p_c, T):
    """Eq. (5): Pi(p) = 1 / (1 + exp((p_c - p) / T))."""
    z = np.clip((p_c - np.asarray(p, dtype=float)) / T, -700.0, 700.0)
    return 1.0 / (1.0 + np.exp(z))


@dataclass
class FDFit:
    p_c: float
    T: float
    p_c_err: float
    T_err: float
    n_points: int


def fit_fermi_dirac(p, k, n) -> FDFit:
    """Binomial maximum-likelihood fit of Eq. (5) to k percolating of n
    configurations at each p.  Errors from the inverse Fisher information."""
    from scipy.optimize import minimize

    p = np.asarray(p, dtype=float)
    k = np.asarray(k, dtype=float)
    n = np.asarray(n, dtype=float)
    if p.size < 2:
        raise ValueError("need at least two values of p")
    frac = k / np.maximum(n, 1.0)

    def nll(theta):
        p_c, logT = theta
        T = np.exp(logT)
        z = (p_c - p) / T
        # log Pi = -log(1 + e^z), log(1 - Pi) = -log(1 + e^-z)
        return float(np.sum(k * np.logaddexp(0.0, z) + (n - k) * np.logaddexp(0.0, -z)))

    # start: p where the empirical curve crosses 1/2, width from its spread
    order = np.argsort(p)
    ps, fs = p[order], frac[order]
    above = np.nonzero(fs >= 0.5)[0]
    p0 = ps[above[0]] if above.size else ps[-1]
    span = max(ps[-1] - ps[0], 1e-3)
    best = None
    for T0 in (span / 50, span / 10, span / 3):
        r = minimize(nll, x0=[p0, np.log(T0)], method="Nelder-Mead",
                     options={"xatol": 1e-10, "fatol": 1e-10, "maxiter": 20000})
        if best is None or r.fun < best.fun:
            best = r
    p_c, T = float(best.x[0]), float(np.exp(best.x[1]))
    # Fisher information of (p_c, T): sum_i n_i (dPi/dtheta)^2 / (Pi (1 - Pi))
    Pi = fermi_dirac(p, p_c, T)
    dPi_dpc = -Pi * (1.0 - Pi) / T
    dPi_dT = Pi * (1.0 - Pi) * (p_c - p) / T**2
    w = n / np.maximum(Pi * (1.0 - Pi), 1e-300)
    I = np.array([[np.sum(w * dPi_dpc**2), np.sum(w * dPi_dpc * dPi_dT)],
                  [np.sum(w * dPi_dpc * dPi_dT), np.sum(w * dPi_dT**2)]])
    try:
        cov = np.linalg.inv(I)
        e_pc, e_T = float(np.sqrt(max(cov[0, 0], 0.0))), float(np.sqrt(max(cov[1, 1], 0.0)))
    except np.linalg.LinAlgError:
        e_pc, e_T = float("inf"), float("inf")
    return FDFit(p_c, T, e_pc, e_T, int(p.size))


@dataclass
class FSSFit:
    p_inf: float
    p_inf_err: float
    slopes: dict  # aspect ratio W/L -> (C, C_err)
    chi2: float
    dof: int


def fit_fss(W, L, p_c, p_c_err, nu: float = NU_3D) -> FSSFit:
    """Eq. (7): joint weighted least squares of p_c(W, L) = p_inf + C(W/L) x,
    x = L^(-1/nu), with one common intercept and one slope per aspect ratio."""
    W = np.asarray(W, dtype=float)
    L = np.asarray(L, dtype=float)
    y = np.asarray(p_c, dtype=float)
    s = np.asarray(p_c_err, dtype=float)
    if np.any(s <= 0):
        raise ValueError("p_c errors must be positive")
    x = L ** (-1.0 / nu)
    ratios = sorted({round(w / l, 12) for w, l in zip(W, L)})
    col = {r: j for j, r in enumerate(ratios)}
    X = np.zeros((y.size, 1 + len(ratios)))
    X[:, 0] = 1.0
    for i, (w, l) in enumerate(zip(W, L)):
        X[i, 1 + col[round(w / l, 12)]] = x[i]
    Xw = X / s[:, None]
    yw = y / s
    beta, *_ = np.linalg.lstsq(Xw, yw, rcond=None)
    cov = np.linalg.pinv(Xw.T @ Xw)
    res = yw - Xw @ beta
    dof = max(y.size - X.shape[1], 0)
    slopes = {r: (float(beta[1 + j]), float(np.sqrt(max(cov[1 + j, 1 + j], 0.0))))
              for r, j in col.items()}
    return FSSFit(float(beta[0]), float(np.sqrt(max(cov[0, 0], 0.0))), slopes,
                  float(res @ res), dof)


def slope_law(r, C0, C1, alpha):
    """Eq. (8): C(W/L) = C0 + C1 (W/L)^alpha."""
    return C0 + C1 * np.asarray(r, dtype=float) ** alpha


def fit_slope_law(r, C, C_err=None):
    """Fit Eq. (8) to the per-aspect-ratio slopes; returns (C0, C1, alpha) and
    their standard errors."""
    from scipy.optimize import curve_fit

    r = np.asarray(r, dtype=float)
    C = np.asarray(C, dtype=float)
    sigma = None if C_err is None else np.asarray(C_err, dtype=float)
    popt, pcov = curve_fit(slope_law, r, C, p0=[0.0, 0.3, -1.2], sigma=sigma,
                           absolute_sigma=sigma is not None, maxfev=20000)
    return tuple(float(v) for v in popt), tuple(float(np.sqrt(max(d, 0.0))) for d in np.diag(pcov))


def p_c_eq9(W, L, p_inf, C0, C1, alpha, nu: float = NU_3D):
    """Eq. (9): effective threshold of a W x L fibre."""
    W = np.asarray(W, dtype=float)
    L = np.asarray(L, dtype=float)
    return p_inf + C0 * L ** (-1.0 / nu) + C1 * W ** alpha * L ** (-alpha - 1.0 / nu)


# ---------------------------------------------------------------------------
# Measurement: Pi(p) curves from the GPU inspection, two passes per size
# ---------------------------------------------------------------------------

COARSE_P = tuple(round(0.08 + 0.02 * i, 2) for i in range(27))  # 0.08 .. 0.60


def measure(specs):
    """Percolating counts of queries [(W, L, p, seed, config_begin, n)], all
    in one batched GPU submission (pc_batch_run).  Only verdicts are needed,
    so the batch propagates the exact reached set alone (PC_BITS_ONLY)."""
    from . import pc_batch_run

    _, res = pc_batch_run(list(specs), device=False, bits_only=True)
    return [r["n_percolating"] for r in res]


def scan(sizes, seed: int, n_coarse: int = 256, n_fine: int = 1024, fine_points: int = 13,
         coarse_p=COARSE_P):
    """Effective thresholds of each (W, L) in ``sizes``: a coarse pass over
    ``coarse_p`` (n_coarse configurations per point) locates the transition;
    a fine pass of ``fine_points`` values over p_c +- 3T (n_fine
    configurations each) is fitted with Eq. (5).  Returns
    {(W, L): (FDFit, p, k, n)} of the fine pass.

    Each fine point inspects its own configurations (j * n_fine onwards for
    point j): the occupancy stream couples the draws of one configuration
    across p, so reusing configurations would make the counts of
    neighbouring points correlated, and the binomial errors of Eq. (5)'s fit
    -- which assume independent counts -- too small."""
    sizes = [tuple(s) for s in sizes]
    specs = [(W, L, p, seed, 0, n_coarse) for (W, L) in sizes for p in coarse_p]
    k = measure(specs)
    fine_specs, grids = [], {}
    for i, (W, L) in enumerate(sizes):
        kk = np.asarray(k[i * len(coarse_p):(i + 1) * len(coarse_p)])
        f = fit_fermi_dirac(coarse_p, kk, np.full(kk.size, n_coarse))
        half = max(3.0 * f.T, 0.01)
        lo, hi = max(f.p_c - half, 1e-4), min(f.p_c + half, 1.0)
        grid = np.round(np.linspace(lo, hi, fine_points), 6)
        grids[(W, L)] = grid
        fine_specs += [(W, L, float(p), seed, j * n_fine, n_fine) for j, p in enumerate(grid)]
    k2 = measure(fine_specs)
    out = {}
    for i, (W, L) in enumerate(sizes):
        kk = np.asarray(k2[i * fine_points:(i + 1) * fine_points])
        nn = np.full(kk.size, n_fine)
        out[(W, L)] = (fit_fermi_dirac(grids[(W, L)], kk, nn), grids[(W, L)], kk, nn)
    return out


def extrapolate(curves, nu: float = NU_3D):
    """Eqs. (7)-(8) over the fitted sizes of ``scan``: p_c_inf, the slope per
    aspect ratio, and the slope law (when at least 3 ratios are present)."""
    keys = sorted(curves)
    W = [k[0] for k in keys]
    L = [k[1] for k in keys]
    pcs = [curves[k][0].p_c for k in keys]
    errs = [max(curves[k][0].p_c_err, 1e-6) for k in keys]
    f = fit_fss(W, L, pcs, errs, nu)
    law = None
    if len(f.slopes) >= 3:
        r = sorted(f.slopes)
        try:
            law = fit_slope_law(r, [f.slopes[x][0] for x in r], [max(f.slopes[x][1], 1e-9) for x in r])
        except RuntimeError:
            law = None
    return f, law


# ---------------------------------------------------------------------------
# Length dependence at fixed width (Sec. III, Fig. 6(a)): Pi ~ exp(-lambda L)
# ---------------------------------------------------------------------------

@dataclass
class DecayFit:
    lam: float      # mean block failure rate lambda_bar: Pi ~ exp(-lambda_bar L)
    lam_err: float
    n_points: int   # lengths with 0 < Pi < 1 used in the fit


def decay_rate(L, k, n) -> DecayFit:
    """Fit ln Pi(L) = c - lambda_bar L (Sec. III: the fibre as a chain of
    blocks, Pi = prod (1 - lambda_i) ~ exp(-lambda_bar L)) by weighted least
    squares over the lengths with 0 < k < n; var(ln Pi) ~ (1 - Pi) / (n Pi)."""
    L = np.asarray(L, dtype=float)
    k = np.asarray(k, dtype=float)
    n = np.asarray(n, dtype=float)
    use = (k > 0) & (k < n)
    if use.sum() < 2:
        # fully percolating (or never) over the range: no measurable decay
        return DecayFit(0.0 if np.all(k == n) else float("inf"), 0.0, int(use.sum()))
    Pi = k[use] / n[use]
    y = np.log(Pi)
    w = n[use] * Pi / (1.0 - Pi)
    X = np.stack([np.ones(use.sum()), -L[use]], axis=1)
    Xw = X * np.sqrt(w)[:, None]
    beta, *_ = np.linalg.lstsq(Xw, y * np.sqrt(w), rcond=None)
    cov = np.linalg.pinv(Xw.T @ Xw)
    return DecayFit(float(beta[1]), float(np.sqrt(max(cov[1, 1], 0.0))), int(use.sum()))


def length_scan(W: int, lengths, ps, n: int, seed: int):
    """Pi(L) at fixed W for each p (one batched submission, verdicts only).
    Returns {p: (L array, k array, n array, DecayFit)}."""
    lengths = [int(L) for L in lengths]
    specs = [(W, L, float(p), seed, 0, n) for p in ps for L in lengths]
    k = np.asarray(measure(specs), dtype=float)
    out = {}
    for i, p in enumerate(ps):
        kk = k[i * len(lengths):(i + 1) * len(lengths)]
        nn = np.full(kk.size, float(n))
        out[float(p)] = (np.asarray(lengths), kk, nn, decay_rate(lengths, kk, nn))
    return out
