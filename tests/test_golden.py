"""The oracle reproduces its stored outputs (tests/golden/make_golden.py wrote them)."""
import json
import os

import numpy as np

import oracle
import scenegen as sg

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_oracle_matches_stored_cfg1_paths():
    with open(os.path.join(HERE, "cfg1_512_paths.json")) as f:
        g = json.load(f)
    r = oracle.render(sg.cfg1_homogeneous_cube(n_paths=512), n_threads=2, path_events=True)
    assert [int(v) for v in r["path_events"]] == g["path_events"]
    # counters added after the fixture was written (interface reflections) are zero here
    assert {k: r["counters"][k] for k in g["counters"]} == g["counters"]
    assert all(v == 0 for k, v in r["counters"].items() if k not in g["counters"])
    assert np.allclose(r["face"].sum(axis=2).ravel(), g["face_total"], rtol=1e-12, atol=1e-15)


def test_oracle_matches_stored_hero_paths():
    with open(os.path.join(HERE, "cfg2_hero4_512_paths.json")) as f:
        g = json.load(f)
    sc = sg.cfg2_cornell_box(width=16, height=16, grid=24, n_paths=512)
    r = oracle.render(sc, n_threads=2, path_events=True, hero=4)
    assert [int(v) for v in r["path_events"]] == g["path_events"]
    assert {k: r["counters"][k] for k in g["counters"]} == g["counters"]
    assert all(v == 0 for k, v in r["counters"].items() if k not in g["counters"])
    for key in ("face", "absorbed", "emitted"):
        assert np.allclose(r[key].ravel(), g[key], rtol=1e-10, atol=1e-15), key
    assert abs(r["film"].sum() - g["film_total"]) <= 1e-10 * abs(g["film_total"])
