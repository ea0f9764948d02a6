"""Calibration of the statistical acceptance rules of the parity tests (`tests/stats.py`): the
oracle against itself, with independent seeds, on the parity tests' main workloads and batch
shapes. Writes `tests/golden/acceptance_calibration.json`, which
`tests/test_acceptance_calibration.py` checks the rules against.

It calls only the oracle and the pure-numpy comparisons of `tests/stats.py` (the same functions
the GPU parity tests call), so the rules are fixed by the oracle's own sampling noise, never by the
CUDA path. Each trial renders a workload with seed s and with seed s + 1000 (the parity tests'
independent seed), in K batches of n paths, and records for every tally:
  - per-bin z-scores: the number of populated bins, those beyond |z| = 3, the largest |z| and the
    reduced chi-square (as `parity_verdict` with the chi-square band, i.e. independent seeds);
  - integrated rows (faces x fluoresced, or dyes): rows beyond max(0.5 %, 3 SE) and 4 SE.

Usage: python tests/golden/calibrate_acceptance.py [--trials N] [--threads T]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import scenegen as sg  # noqa: E402
from tests.stats import bin_parity, integrated_independent  # noqa: E402

# name -> (scene, batches K, paths per batch, oracle settings); the shapes of
# tests/test_gpu_parity.py::test_cfg1_homogeneous_cube_parity and ::test_cfg2_*_reduced_parity
WORKLOADS = {
    "cfg1_homogeneous_cube": (lambda: sg.cfg1_homogeneous_cube(n_paths=100_000), 32, 100_000 // 32, {}),
    "cfg2_cornell_box_48": (lambda: sg.cfg2_cornell_box(width=48, height=48, grid=48, n_paths=1), 32, 6000,
                            {"skip_cell": 1}),
}
KEYS = ("face", "absorbed", "emitted", "film")


def run(sc, K, n, seed, threads, kw):
    return [oracle.render(sc, n_paths=n, path_offset=k * n, seed=seed, n_threads=threads, **kw)
            for k in range(K)]


def trial(sc, K, n, seed, threads, kw):
    a = run(sc, K, n, seed, threads, kw)
    b = run(sc, K, n, seed + 1000, threads, kw)
    out = {}
    for key in KEYS:
        if a[0].get(key) is None:
            continue
        v = bin_parity(a, b, key, same_seed=False)
        n_bins = v["n"]
        rec = {"bins": n_bins, "bins_over_3": int(round(v.get("frac_gt3", 0.0) * n_bins)),
               "max_abs_z": v.get("max_abs_z", 0.0), "red_chi2": v.get("red_chi2", 0.0), "ok": bool(v["ok"])}
        if key != "film":
            ok, info = integrated_independent(a, b, key)
            rec.update({"rows": info["rows"], "rows_over_3se": info["rows_over_3se"],
                        "rows_over_4se": info["rows_over_4se"], "integrated_ok": bool(ok)})
        out[key] = rec
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--trials", type=int, default=12)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "acceptance_calibration.json"))
    args = ap.parse_args()
    res = {"description": "oracle vs oracle, independent seeds (s, s + 1000), per-bin z and "
                          "integrated rows as the parity tests compute them",
           "script": "tests/golden/calibrate_acceptance.py", "trials": args.trials, "workloads": {}}
    for name, (make, K, n, kw) in WORKLOADS.items():
        sc = make()
        t0 = time.time()
        trials = [trial(sc, K, n, 101 + 7 * t, args.threads, kw) for t in range(args.trials)]
        res["workloads"][name] = {"K": K, "paths_per_batch": n, "settings": kw, "seeds": [101 + 7 * t for t in range(args.trials)],
                                  "seconds": round(time.time() - t0, 1), "trials": trials}
        print(name, f"{time.time() - t0:.0f} s", flush=True)
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
