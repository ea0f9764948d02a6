"""Batched persistent form: many independent media in one launch (C ABI, sm_103a).

Medium m of a batch draws its random numbers under (seed, medium_id + m), so it must reproduce,
bit for bit in the fixed-point tallies, a single-scene render of that medium with that medium id.
The single-scene kernels are in turn checked against the oracle (test_gpu_parity.py); the oracle
is also compared directly on integrated tallies here.
"""
import numpy as np
import pytest

import oracle
import scenegen as sg
from paper_1706_03024_gb300 import native as N
from paper_1706_03024_gb300.scene import Batch, Scene
from tests.gpu_common import compare_integrated, require_gpu

pytestmark = pytest.mark.gpu

MD = N.FLR_MAX_DYES_PER_MEDIUM


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def single_tallies(sc, medium_id, seed, form="plain"):
    S = Scene(sc)
    S.render(medium_id=medium_id, seed=seed, form=form, film=False)
    r = S.read()
    S.close()
    return r


def assert_medium_equal(batch_out, m, single, D):
    assert np.array_equal(batch_out["face"][m], single["face"]), m
    assert np.array_equal(batch_out["absorbed"][m, :D + 1], single["absorbed"]), m
    assert not batch_out["absorbed"][m, D + 1:].any()
    assert np.array_equal(batch_out["emitted"][m, :D], single["emitted"]), m


def test_batch_equals_single_scene_per_medium():
    media = sg.cfg3_batched_media(n_media=12, seed=0, max_edge=32, path_scale=0.02)
    bt = Batch(media, seed=5, medium_id=100)
    bt.launch()
    out = bt.read()
    tot = {k: 0 for k in N.COUNTER_NAMES}
    for m, sc in enumerate(media):
        s = single_tallies(sc, 100 + m, 5)
        assert_medium_equal(out, m, s, sc["dyes"]["eps"].shape[0])
        for k, v in s["counters"].items():
            tot[k] += v
    for k in ("paths", "events", "nulls", "escapes", "absorbed_dead", "rr_kills", "cap_hits",
              "emissions", "dye_absorptions", "scatters", "steps"):
        assert out["counters"][k] == tot[k], k
    assert out["counters"]["paths"] == int(bt.n_paths.sum())


def test_batch_graph_replay_is_deterministic():
    media = sg.cfg3_batched_media(n_media=8, seed=1, max_edge=24, path_scale=0.02)
    bt = Batch(media, seed=9)
    bt.launch()
    a = bt.read()
    bt.launch()
    b = bt.read()
    for key in ("face", "absorbed", "emitted"):
        assert np.array_equal(a[key], b[key])
    assert a["counters"] == b["counters"]


def test_batch_matches_oracle_integrated():
    media = sg.cfg3_batched_media(n_media=5, seed=2, max_edge=20, path_scale=0.05)
    for sc in media:
        sc["params"]["n_paths"] = 20_000
    bt = Batch(media, seed=0, medium_id=0)
    bt.launch()
    out = bt.read()
    for m, sc in enumerate(media):
        D = sc["dyes"]["eps"].shape[0]
        o = oracle.render(sc, medium_id=m, seed=0)
        assert compare_integrated(out["face"][m].sum(-1), o["face"].sum(-1)) <= 5e-3, m
        assert compare_integrated(out["absorbed"][m, :D + 1].sum(-1), o["absorbed"].sum(-1)) <= 5e-3
        assert compare_integrated(out["emitted"][m, :D].sum(-1), o["emitted"].sum(-1)) <= 5e-3


def test_batch_uneven_sizes_and_homogeneous_media():
    media = sg.cfg3_batched_media(n_media=4, seed=3, max_edge=16, path_scale=0.01)
    # one homogeneous medium (no grids), one with a single path, one with zero paths
    h = sg.cfg1_homogeneous_cube(n_paths=3000)
    h["sensor"] = sg.no_sensor()
    media.append(h)
    media[0]["params"]["n_paths"] = 1
    media[1]["params"]["n_paths"] = 0
    bt = Batch(media, seed=4, medium_id=7)
    bt.launch()
    out = bt.read()
    assert not out["face"][1].any()
    for m in (0, 2, 3, 4):
        s = single_tallies(media[m], 7 + m, 4)
        assert_medium_equal(out, m, s, media[m]["dyes"]["eps"].shape[0])


def test_batch_full_size_sampled_media():
    """The 256-medium workload at full path counts (the benchmarked launch): invariants on every
    medium and bit-identity with single-scene renders on sampled media."""
    media = sg.cfg3_batched_media(n_media=256, seed=0)
    bt = Batch(media, seed=0, medium_id=0)
    bt.launch()
    out = bt.read()
    c = out["counters"]
    n = int(bt.n_paths.sum())
    ends = (c["escapes"] + c["absorbed_dead"] + c["rr_kills"] + c["cap_hits"] + c["step_budget"]
            + c["vf_rejected"])
    assert c["paths"] == n and ends == n
    assert c["majorant_violations"] == 0 and c["nonfinite"] == 0 and c["step_budget"] == 0
    face_tot = out["face"].sum(axis=(1, 2, 3))
    assert (face_tot <= 1.0 + 1e-9).all() and (face_tot >= 0).all()
    rng = np.random.default_rng(0)
    for m in rng.choice(256, size=3, replace=False):
        m = int(m)
        s = single_tallies(media[m], m, 0, form="wavefront")
        assert_medium_equal(out, m, s, media[m]["dyes"]["eps"].shape[0])


def test_batch_rejects_bad_media():
    media = sg.cfg3_batched_media(n_media=2, seed=4, max_edge=16, path_scale=0.01)
    media[1]["sources"] = [sg.pencil_beam((0.5, 0.5, 0.0), (0, 0, 1), [450.0] * 8),
                           sg.pencil_beam((0.5, 0.5, 0.0), (0, 0, 1), [460.0])]
    with pytest.raises(N.FluoroError) as e:
        Batch(media)
    assert e.value.code == N.FLR_ERR_ARG


def test_batch_per_bin_parity_with_the_oracle():
    """Four media of the batched workload, each traced by the batch and by the oracle over 16 batches
    of the same path ids (the batch draws medium m's numbers under medium id m): per-bin parity of
    the face, absorbed and emitted tallies by batch means (at most 1 % of populated bins beyond
    |z| = 3, none beyond 5.5), the same-seed integrated tallies within 0.5 %, and every path's tally
    in the same medium as the single-scene kernel's."""
    from tests.gpu_common import bin_parity, paired_integrated
    media = sg.cfg3_batched_media(n_media=4, seed=6, max_edge=24)
    K, n = 16, 2000
    for sc in media:
        sc["params"]["n_paths"] = n
    g = {m: [] for m in range(len(media))}
    for k in range(K):
        bt = Batch(media, seed=0, medium_id=0, path_offset=k * n)
        bt.launch()
        out = bt.read()
        for m, sc in enumerate(media):
            D = sc["dyes"]["eps"].shape[0]
            g[m].append({"face": out["face"][m], "absorbed": out["absorbed"][m, :D + 1],
                         "emitted": out["emitted"][m, :D]})
        bt.close()
    for m, sc in enumerate(media):
        o = [oracle.render(sc, n_paths=n, path_offset=k * n, medium_id=m, seed=0, film=False)
             for k in range(K)]
        for key in ("face", "absorbed", "emitted"):
            v = bin_parity(g[m], o, key)
            assert v["ok"], (m, key, v)
            ok, worst, _, info = paired_integrated(g[m], o, key)
            assert ok, (m, key, worst, info)
