"""Writes the stored oracle outputs under tests/golden/ (calls only oracle/ and scenegen).

Run from the repository root:  python tests/golden/make_golden.py
The fixture pins the oracle against accidental drift (tests/test_golden.py) and gives the GPU
parity tests per-path event counts to measure how often the two sides take identical paths.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import scenegen as sg  # noqa: E402


def main():
    sc = sg.cfg1_homogeneous_cube(n_paths=512)
    r = oracle.render(sc, n_threads=1, path_events=True)
    out = {
        "scene": "cfg1_homogeneous_cube (scenegen), seed 0, paths 0..511, weighted QY mode",
        "path_events": [int(v) for v in r["path_events"]],
        "counters": r["counters"],
        "face_total": [float(v) for v in r["face"].sum(axis=2).ravel()],
        "emitted_total": float(r["emitted"].sum()),
    }
    with open(os.path.join(HERE, "cfg1_512_paths.json"), "w") as f:
        json.dump(out, f, indent=1)

    # hero-wavelength paths (four members) on a small Cornell box
    sc = sg.cfg2_cornell_box(width=16, height=16, grid=24, n_paths=512)
    r = oracle.render(sc, n_threads=1, path_events=True, hero=4)
    out = {
        "scene": "cfg2_cornell_box(width=16, height=16, grid=24) (scenegen), seed 0, paths 0..511, hero 4",
        "path_events": [int(v) for v in r["path_events"]],
        "counters": r["counters"],
        "face": [float(v) for v in r["face"].ravel()],
        "absorbed": [float(v) for v in r["absorbed"].ravel()],
        "emitted": [float(v) for v in r["emitted"].ravel()],
        "film_total": float(r["film"].sum()),
    }
    with open(os.path.join(HERE, "cfg2_hero4_512_paths.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
