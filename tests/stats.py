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


# ---------------------------------------------------------------------------------------------
# Comparisons of batched tallies (lists of per-batch result dicts), shared by the GPU parity tests
# and the acceptance calibration (tests/golden/calibrate_acceptance.py).

def totals(outs, key):
    return np.sum([o[key] for o in outs], axis=0) / len(outs)


def compare_integrated(g, o, rel=5e-3, floor=1e-3):
    """Same-seed integrated tallies: relative difference <= rel where the value is at least
    `floor` of the largest; returns the worst relative difference."""
    g, o = np.asarray(g, np.float64), np.asarray(o, np.float64)
    big = np.abs(o) >= floor * max(np.abs(o).max(), 1e-300)
    worst = 0.0
    if big.any():
        worst = float((np.abs(g[big] - o[big]) / np.abs(o[big])).max())
    return worst


def bin_parity(g_outs, o_outs, key, min_nonzero=None, same_seed=True):
    gs = np.stack([x[key] for x in g_outs])
    os_ = np.stack([x[key] for x in o_outs])
    K = gs.shape[0]
    if min_nonzero is None:
        min_nonzero = (3 * K) // 4
    mg, sg = batch_mean_se(gs)
    mo, so = batch_mean_se(os_)
    populated = ((gs != 0).sum(axis=0) >= min_nonzero) & ((os_ != 0).sum(axis=0) >= min_nonzero)
    sg = np.where(populated, sg, 0.0)
    so = np.where(populated, so, 0.0)
    return parity_verdict(mg, sg, mo, so, check_chi2=not same_seed)


def integrated_independent(g_outs, o_outs, key, rel=5e-3):
    """Independent seeds: per-row totals agree within max(rel, 3 SE). With a dozen rows (faces x
    fluoresced) one row beyond 3 SE is expected about 3 % of the time, so one is allowed as long as
    none is beyond max(rel, 4 SE)."""
    gs = np.stack([x[key].sum(axis=-1) for x in g_outs])
    os_ = np.stack([x[key].sum(axis=-1) for x in o_outs])
    mg, sg = batch_mean_se(gs)
    mo, so = batch_mean_se(os_)
    se = np.sqrt(sg ** 2 + so ** 2)
    big = np.abs(mo) >= 1e-3 * max(np.abs(mo).max(), 1e-300)
    d = np.abs(mg - mo)
    over3 = (d > np.maximum(rel * np.abs(mo), 3.0 * se)) & big
    over4 = (d > np.maximum(rel * np.abs(mo), 4.0 * se)) & big
    ok = int(over3.sum()) <= 1 and not over4.any()
    return ok, {"gpu": mg[big].tolist()[:12], "oracle": mo[big].tolist()[:12], "rows": int(big.sum()),
                "rows_over_3se": int(over3.sum()), "rows_over_4se": int(over4.sum())}


def paired_integrated(g_outs, o_outs, key, rel=5e-3, z=4.0, floor=1e-3):
    """Same seed, same path ids, batch by batch: the GPU and the oracle trace nearly the same
    paths, so their integrated tallies (per row: face x fluoresced, or dye) differ only through the
    paths whose fp32 and fp64 trajectories part. With d_k = gpu_k - oracle_k over K batches of the
    same path ids and SE_d its standard error, a row passes if |mean d| <= rel |oracle| (0.5 %);
    a row whose paired standard error is too large for that test to mean anything (z SE_d above
    rel |oracle|) must instead satisfy |mean d| <= z SE_d. Returns (ok, worst relative difference
    over the precise rows, number of precise rows, details)."""
    gs = np.stack([x[key].sum(axis=-1) for x in g_outs]).reshape(len(g_outs), -1)
    os_ = np.stack([x[key].sum(axis=-1) for x in o_outs]).reshape(len(o_outs), -1)
    d = gs - os_
    md, sd = batch_mean_se(d)
    mo = os_.mean(axis=0)
    big = np.abs(mo) >= floor * max(np.abs(mo).max(), 1e-300)
    precise = big & (z * sd <= rel * np.abs(mo))
    loose = big & ~precise
    ok = bool(np.all(np.abs(md[precise]) <= rel * np.abs(mo[precise])) and
              np.all(np.abs(md[loose]) <= z * sd[loose]))
    worst = float((np.abs(md[precise]) / np.abs(mo[precise])).max()) if precise.any() else 0.0
    return ok, worst, int(precise.sum()), {"mean_diff": md[big].tolist(), "se": sd[big].tolist(),
                                           "oracle": mo[big].tolist()}
