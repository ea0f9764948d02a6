"""The statistical acceptance rules of the parity tests against their calibration: the oracle
compared with itself under independent seeds (`tests/golden/calibrate_acceptance.py`, output
`tests/golden/acceptance_calibration.json`). The rules must accept nearly every such comparison
(there is no difference to find), and the stored trials must have been taken with the rules and
the batch shapes the parity tests use now."""
from __future__ import annotations

import inspect
import json
import os

import pytest

from tests import stats

HERE = os.path.dirname(os.path.abspath(__file__))
CAL = os.path.join(HERE, "golden", "acceptance_calibration.json")


def _load():
    with open(CAL) as f:
        return json.load(f)


def _defaults():
    sig = inspect.signature(stats.parity_verdict)
    return {k: v.default for k, v in sig.parameters.items() if v.default is not inspect.Parameter.empty}


def _per_bin_ok(rec, d):
    """parity_verdict's decision, from a trial's summary numbers."""
    n, n3 = rec["bins"], rec["bins_over_3"]
    if n == 0:
        return True
    ok = (n3 / n <= d["frac_limit"] or n3 <= 3) and rec["max_abs_z"] <= d["max_limit"]
    if n >= d["min_bins"]:
        ok = ok and d["chi_lo"] <= rec["red_chi2"] <= d["chi_hi"]
    return ok


def _strict_ok(rec, d):
    """The same rule without the three-bin allowance (at most 1 % of the bins beyond |z| = 3)."""
    n, n3 = rec["bins"], rec["bins_over_3"]
    if n == 0:
        return True
    ok = n3 / n <= d["frac_limit"] and rec["max_abs_z"] <= d["max_limit"]
    if n >= d["min_bins"]:
        ok = ok and d["chi_lo"] <= rec["red_chi2"] <= d["chi_hi"]
    return ok


def test_calibration_was_taken_on_the_parity_tests_shapes():
    cal = _load()
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "calibrate_acceptance", os.path.join(HERE, "golden", "calibrate_acceptance.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert set(cal["workloads"]) == set(mod.WORKLOADS)
    for name, (_, K, n, kw) in mod.WORKLOADS.items():
        w = cal["workloads"][name]
        assert (w["K"], w["paths_per_batch"], w["settings"]) == (K, n, kw), name
        assert len(w["trials"]) == cal["trials"] >= 50


def test_recorded_decisions_are_the_current_rules():
    """A change of the limits in tests/stats.py without a new calibration fails here."""
    d = _defaults()
    for name, w in _load()["workloads"].items():
        for t in w["trials"]:
            for key, rec in t.items():
                assert _per_bin_ok(rec, d) == rec["ok"], (name, key, rec)
                if "rows" in rec:
                    ok = rec["rows_over_3se"] <= 1 and rec["rows_over_4se"] == 0
                    assert ok == rec["integrated_ok"], (name, key, rec)


@pytest.mark.parametrize("key", ["face", "absorbed", "emitted", "film"])
def test_per_bin_rule_accepts_oracle_against_itself(key):
    """False-failure rate of the per-bin rule on identical estimators: at most 3 % per tally."""
    d = _defaults()
    for name, w in _load()["workloads"].items():
        recs = [t[key] for t in w["trials"] if key in t]
        if not recs:
            continue
        fails = sum(not _per_bin_ok(r, d) for r in recs)
        assert fails <= 0.03 * len(recs), (name, key, fails, len(recs))


def test_integrated_rule_accepts_oracle_against_itself():
    for name, w in _load()["workloads"].items():
        for key in ("face", "absorbed", "emitted"):
            recs = [t[key] for t in w["trials"] if key in t and "rows" in t[key]]
            fails = sum(not r["integrated_ok"] for r in recs)
            assert fails <= 0.03 * len(recs), (name, key, fails, len(recs))


def test_three_bin_allowance_is_needed_and_no_looser_than_needed():
    """Spectral tallies have tens of bins: the strict 1 % rule (no bin beyond |z| = 3 below 100
    bins) rejects a visible share of identical-estimator comparisons, which the three-bin
    allowance removes; and no trial needed more than three bins."""
    d = _defaults()
    strict_fails, total, worst = 0, 0, 0
    for w in _load()["workloads"].values():
        for t in w["trials"]:
            for key in ("face", "absorbed", "emitted"):
                if key not in t:
                    continue
                r = t[key]
                total += 1
                strict_fails += not _strict_ok(r, d)
                if r["bins"] < 300:
                    worst = max(worst, r["bins_over_3"])
    assert strict_fails >= 0.02 * total, (strict_fails, total)
    assert worst <= 3, worst
