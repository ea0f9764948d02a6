"""GPU hero-wavelength paths (k_trace_hero through flr_render, hero = C) against the oracle's.

With one member the kernel is the single-wavelength plain kernel: same paths, identical
fixed-point tallies and counters. With four, the GPU and the oracle trace the same paths with the
same seeds (per-path event counts compared), and every spectral tally and the film agree bin by
bin and integrated; the oracle's hero estimator is itself pinned against closed forms and the
single-wavelength estimator (test_oracle_hero.py).
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from paper_1706_03024_gb300 import native as N
from paper_1706_03024_gb300.scene import Scene
from tests.gpu_common import bin_parity, compare_integrated, require_gpu, totals
from tests.test_oracle_hero import ragged_spectrum_scene, two_beams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def workloads():
    return [
        ("homogeneous cube", sg.cfg1_homogeneous_cube(n_paths=1), {}),
        ("cornell box", sg.cfg2_cornell_box(width=24, height=24, grid=32, n_paths=1), {}),
        ("cornell box, leaps", sg.cfg2_cornell_box(width=24, height=24, grid=32, n_paths=1),
         {"skip_cell": 2}),
        ("light sheet", sg.cfg5_light_sheet(grid=32, width=24, height=24, n_blobs=40, n_paths=1,
                                            sigma_t_ref=20.0), {}),
        ("two beams", two_beams(2.0, [0.7, 0.5]), {}),
        ("cornell box, analog, one re-emission",
         sg.cfg2_cornell_box(width=24, height=24, grid=32, n_paths=1),
         {"analog": 1, "max_inelastic": 1}),
        ("ten bins, ragged blocks, five lines", ragged_spectrum_scene(), {}),
    ]


def _fixed(x):
    return np.round(np.asarray(x, np.float64) * 2.0 ** 24).astype(np.int64)


@pytest.mark.parametrize("case", range(7))
def test_one_member_is_the_plain_kernel(case):
    name, sc, kw = workloads()[case]
    S = Scene(sc)
    n = 20000
    pa = torch.zeros(n, dtype=torch.int32, device="cuda")
    pb = torch.zeros(n, dtype=torch.int32, device="cuda")
    fa = S.render(n_paths=n, form="plain", path_events=pa, **kw)
    fa = fa.clone() if fa is not None else None
    a = S.read()
    fb = S.render(n_paths=n, form="plain", hero=1, path_events=pb, **kw)
    b = S.read()
    assert torch.equal(pa, pb), name
    for key in ("face", "absorbed", "emitted"):
        assert np.array_equal(_fixed(a[key]), _fixed(b[key])), (name, key)
    assert a["counters"] == b["counters"], name
    if fa is not None:
        # same contributions, atomics in another order
        assert torch.allclose(fa, fb, rtol=1e-5, atol=1e-7 * float(fa.abs().max())), name


@pytest.mark.parametrize("case", range(7))
def test_hero_matches_oracle_hero(case):
    name, sc, kw = workloads()[case]
    K, n = 16, 2500
    o = [oracle.render(sc, n_paths=n, path_offset=k * n, hero=4, path_events=True, **kw)
         for k in range(K)]
    S = Scene(sc)
    pe = torch.zeros(K * n, dtype=torch.int32, device="cuda")
    g = []
    for k in range(K):
        f = S.render(n_paths=n, path_offset=k * n, form="plain", hero=4,
                     path_events=pe[k * n:(k + 1) * n], **kw)
        r = S.read()
        r["film"] = f.double().cpu().numpy() if f is not None else None
        g.append(r)
    same = float((pe.cpu().numpy().astype(np.uint32)
                  == np.concatenate([x["path_events"] for x in o])).mean())
    assert same >= 0.95, (name, same)
    for key in ("face", "absorbed", "emitted"):
        v = bin_parity(g, o, key)
        assert v["ok"], (name, key, v)
        worst = compare_integrated(totals(g, key).sum(axis=-1), totals(o, key).sum(axis=-1))
        assert worst <= 5e-3, (name, key, worst)
    if sc["sensor"]["kind"] != "none":
        v = bin_parity(g, o, "film")
        assert v["ok"], (name, "film", v)
        # the GPU estimates each connection's transmittance by ratio tracking, the oracle takes
        # it exactly: same expectation, different noise
        gf, of = totals(g, "film").sum(), totals(o, "film").sum()
        se = np.sqrt(np.var([x["film"].sum() for x in g]) / K + np.var([x["film"].sum() for x in o]) / K)
        assert abs(gf - of) <= 5e-3 * of + 4 * se, (name, gf, of, se)
    c = g[-1]["counters"]
    for cn in ("majorant_violations", "nonfinite", "connect_budget", "step_budget"):
        assert c[cn] == 0, (name, cn, c[cn])


BENCH_LAUNCH = {"form": "wavefront_warp", "block_size": 128, "regroup": 1}


@pytest.mark.parametrize("case", range(7))
def test_warp_form_equals_plain_form(case):
    """The warp-regrouped hero kernel traces the same paths and marches as the plain one: identical
    fixed-point tallies, counters and per-path event counts, the same film (fixed-point sums); with
    one member it is the single-wavelength warp kernel."""
    name, sc, kw = workloads()[case]
    S = Scene(sc)
    n = 30000
    for hero, ref in ((4, {"form": "plain", "hero": 4}), (1, dict(BENCH_LAUNCH))):
        pa = torch.zeros(n, dtype=torch.int32, device="cuda")
        pb = torch.zeros(n, dtype=torch.int32, device="cuda")
        fa = S.render(n_paths=n, path_events=pa, **ref, **kw)
        fa = fa.clone() if fa is not None else None
        a = S.read()
        fb = S.render(n_paths=n, path_events=pb, hero=hero, **BENCH_LAUNCH, **kw)
        b = S.read()
        assert torch.equal(pa, pb), (name, hero)
        for key in ("face", "absorbed", "emitted"):
            assert np.array_equal(_fixed(a[key]), _fixed(b[key])), (name, hero, key)
        assert a["counters"] == b["counters"], (name, hero)
        if fa is not None:
            assert torch.allclose(fa, fb, rtol=1e-4, atol=1e-6 * float(fa.abs().max())), (name, hero)


def test_hero_full_size_cornell_box_invariants():
    """The Cornell-box workload at full size (4,194,304 paths, 512 x 512 x 81 film) with four
    wavelengths per path in the benchmarked launch shape: bookkeeping, a finite non-negative
    film, tallies within 1 % of the single-wavelength kernel's on the same path ids."""
    sc = sg.cfg2_cornell_box()
    n = sc["params"]["n_paths"]
    S = Scene(sc)
    film = S.render(hero=4, skip_cell=1, **BENCH_LAUNCH)
    h = S.read()
    c = h["counters"]
    ends = (c["escapes"] + c["absorbed_dead"] + c["rr_kills"] + c["cap_hits"] + c["step_budget"]
            + c["vf_rejected"])
    assert c["paths"] == n and ends == n
    for cn in ("majorant_violations", "nonfinite", "connect_budget", "step_budget"):
        assert c[cn] == 0, cn
    f = film.double()
    assert torch.isfinite(f).all() and (f >= 0).all()
    hf = float(f.sum())
    S.render(form="wavefront_warp", block_size=128, regroup=1, skip_cell=1)
    s1 = S.read()
    sf = float(S.film_tensor().double().sum())
    assert abs(hf - sf) <= 1e-2 * sf, (hf, sf)
    for key in ("face", "emitted"):
        assert abs(h[key].sum() - s1[key].sum()) <= 1e-2 * s1[key].sum(), key


def test_hero_rejects_unsupported_combinations():
    sc = sg.cfg2_cornell_box(width=16, height=16, grid=16, n_paths=1000)
    S = Scene(sc)
    for kw in ({"hero": 5}, {"hero": -1}, {"hero": 4, "form": "wavefront"},
               {"hero": 4, "form": "wavefront_warp", "macro_cell": 4},
               {"hero": 4, "form": "plain", "macro_cell": 4},
               {"hero": 4, "form": "plain", "paper_mode": True}):
        p = S._params(1000, **{k: v for k, v in kw.items() if k != "form"},
                      form=kw.get("form", "plain"))
        p.film = S.film_tensor().data_ptr()
        assert N.flr_render(S.ctx, p, 0) == N.FLR_ERR_ARG, kw
    p = S._params(65536, form="wavefront_warp", hero=4)
    p.film = S.film_tensor().data_ptr()
    assert N.flr_render_camera(S.ctx, p, 0) == N.FLR_ERR_ARG
    assert S.status() == N.FLR_OK
