"""Helpers for the GPU parity tests: run the CUDA path and the oracle on the same path ids."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1706_03024_gb300 import build as B
from paper_1706_03024_gb300.scene import Scene
from tests.stats import (batch_mean_se, bin_parity, compare_integrated,  # noqa: F401
                         integrated_independent, paired_integrated, parity_verdict, totals)


def require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for -m gpu tests (there is no CPU path)")
    B.build()


def gpu_batches(scene, K, n_per, form="plain", scene_obj=None, film=True, **kw):
    S = scene_obj or Scene(scene)
    outs = []
    for k in range(K):
        f = S.render(n_paths=n_per, path_offset=k * n_per, form=form, film=film, **kw)
        r = S.read()
        r["film"] = f.double().cpu().numpy() if (f is not None and film) else None
        outs.append(r)
    return outs


def oracle_batches(scene, K, n_per, film=True, **kw):
    return [oracle.render(scene, n_paths=n_per, path_offset=k * n_per, film=film, **kw)
            for k in range(K)]


def check_workload(sc, K, n_per, forms=("plain",), film_min_nonzero=None, path_id_frac=0.99,
                   launch=None, **kw):
    """GPU against the oracle on the same path ids, K batches of n_per paths: the fraction of paths
    with identical event counts, per-bin parity of the face, absorbed and emitted tallies and the
    film, same-seed integrated tallies within 0.5 %, and an independent seed with the full
    statistical criteria. kw: estimator settings both sides take; launch: GPU launch shape (block
    size, regroup). Returns the same-seed GPU batches per form."""
    launch = launch or {}
    o = oracle_batches(sc, K, n_per, path_events=True, **kw)
    o_events = np.concatenate([x["path_events"] for x in o])
    S = Scene(sc)
    results = {}
    for form in forms:
        pe = torch.zeros(K * n_per, dtype=torch.int32, device="cuda")
        g = []
        for k in range(K):
            f = S.render(n_paths=n_per, path_offset=k * n_per, form=form,
                         path_events=pe[k * n_per:(k + 1) * n_per], **launch, **kw)
            r = S.read()
            r["film"] = f.double().cpu().numpy() if f is not None else None
            g.append(r)
        g_events = pe.cpu().numpy().astype(np.uint32)
        same = float((g_events == o_events).mean())
        assert same >= path_id_frac, (form, same)
        for key in ("face", "absorbed", "emitted"):
            v = bin_parity(g, o, key)
            assert v["ok"], (form, key, v)
            worst = compare_integrated(totals(g, key).sum(axis=-1), totals(o, key).sum(axis=-1))
            assert worst <= 5e-3, (form, key, worst)
        if sc["sensor"]["kind"] != "none":
            v = bin_parity(g, o, "film", film_min_nonzero)
            assert v["ok"], (form, "film", v)
            gf, of = totals(g, "film"), totals(o, "film")
            assert abs(gf.sum() - of.sum()) <= 5e-3 * of.sum() + 4 * np.sqrt(
                np.var([x["film"].sum() for x in g]) / K + np.var([x["film"].sum() for x in o]) / K)
        c = g[-1]["counters"]
        for name in ("majorant_violations", "nonfinite", "connect_budget", "step_budget"):
            assert c[name] == 0, (form, name, c[name])
        results[form] = g
        # independent seed: the full statistical criteria
        seed2 = int(sc["params"]["seed"]) + 1000
        gi = []
        for k in range(K):
            f = S.render(n_paths=n_per, path_offset=k * n_per, form=form, seed=seed2, **launch,
                         **kw)
            r = S.read()
            r["film"] = f.double().cpu().numpy() if f is not None else None
            gi.append(r)
        for key in ("face", "absorbed", "emitted"):
            v = bin_parity(gi, o, key, same_seed=False)
            assert v["ok"], (form, "independent", key, v)
            ok, info = integrated_independent(gi, o, key)
            assert ok, (form, "independent", key, info)
        if sc["sensor"]["kind"] != "none":
            v = bin_parity(gi, o, "film", film_min_nonzero, same_seed=False)
            assert v["ok"], (form, "independent", "film", v)
    return results
