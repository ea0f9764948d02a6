"""Statistical helpers shared by the oracle pins and the GPU parity tests (no method arithmetic)."""
from __future__ import annotations

import math

import numpy as np


def batch_mean_se(samples):
    """samples: array [K, ...] of independent batch estimates -> (mean, standard error)."""
    s = np.asarray(samples, dtype=np.float64)
    K = s.shape[0]
    return s.mean(axis=0), s.std(axis=0, ddof=1) / math.sqrt(K)


def binomial_se(p, n):
    return math.sqrt(max(p * (1.0 - p), 1e-300) / n)


def chi2_counts(observed, expected_prob, min_expected=5.0):
    """Pearson chi-square of integer counts against probabilities; bins with small expectation
    are pooled into one. Returns (chi2, dof)."""
    obs = np.asarray(observed, dtype=np.float64)
    n = obs.sum()
    exp = np.asarray(expected_prob, dtype=np.float64) * n
    big = exp >= min_expected
    o = list(obs[big])
    e = list(exp[big])
    if (~big).any():
        o.append(obs[~big].sum())
        e.append(exp[~big].sum())
    o, e = np.array(o), np.array(e)
    keep = e > 0
    chi2 = float(((o[keep] - e[keep]) ** 2 / e[keep]).sum())
    return chi2, int(keep.sum() - 1)


def chi2_ok(chi2, dof, z=4.0):
    """Accept if chi2 is within z standard deviations of its mean (Wilson-Hilferty)."""
    if dof <= 0:
        return True
    x = (chi2 / dof) ** (1.0 / 3.0)
    mu = 1.0 - 2.0 / (9.0 * dof)
    sd = math.sqrt(2.0 / (9.0 * dof))
    return abs((x - mu) / sd) <= z


def zscores(a, se_a, b, se_b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    se = np.sqrt(np.asarray(se_a, np.float64) ** 2 + np.asarray(se_b, np.float64) ** 2)
    mask = se > 0
    z = np.zeros_like(a)
    z[mask] = (a[mask] - b[mask]) / se[mask]
    return z, mask


def parity_verdict(a, se_a, b, se_b, frac_limit=0.01, max_limit=5.5, chi_lo=0.8, chi_hi=1.2,
                   min_bins=500, check_chi2=True):
    """Per-bin agreement criteria: fraction of |z| > 3 at most frac_limit, max |z| at most
    max_limit and, when enough bins are populated, reduced chi-square in [chi_lo, chi_hi].
    The chi-square band assumes independent estimates: runs that share their random numbers
    (same seed, same path ids) agree far better than their standard errors, so for them only the
    |z| limits apply (check_chi2=False). The band also needs many weakly correlated bins: the
    bins of one spectral tally move together (a dye's emission row scales with its total), so
    mean z^2 over a few dozen of them behaves like a chi-square with few degrees of freedom; it is
    applied from min_bins = 500 populated bins on (films)."""
    z, m = zscores(a, se_a, b, se_b)
    zz = z[m]
    if zz.size == 0:
        return {"ok": True, "n": 0}
    n_gt3 = int((np.abs(zz) > 3).sum())
    frac = n_gt3 / zz.size
    zmax = float(np.abs(zz).max())
    red = float((zz ** 2).mean())
    # a spectral tally has tens of bins, and z from K batch means has t-like tails that cluster
    # over neighbouring bins: up to 3 bins beyond 3 are accepted whatever the bin count
    ok = (frac <= frac_limit or n_gt3 <= 3) and zmax <= max_limit
    if check_chi2 and zz.size >= min_bins:
        ok = ok and chi_lo <= red <= chi_hi
    return {"ok": ok, "n": int(zz.size), "frac_gt3": frac, "max_abs_z": zmax, "red_chi2": red}
