"""GPU (C ABI, sm_103a kernels) against the CPU oracle on the same seeded inputs.

Criteria: per spectral bin and per pixel, z = (gpu - oracle) / sqrt(SE_gpu^2 + SE_oracle^2) from
K batch means (batches = disjoint path-id ranges): at most 1 % of populated bins beyond 3, none
beyond 5.5. Two runs per workload: with the oracle's seed (nearly identical paths: integrated
tallies within 0.5 % relative, and the fraction of paths with identical event counts reported and
bounded), and with an independent seed (adds reduced chi-square in [0.8, 1.2] when >= 500 bins
are populated, i.e. on films, and integrated tallies within max(0.5 %, 3 SE)). Bit-exact where the work is integer:
Philox blocks, emission bins, fixed-point tallies between launch forms.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from paper_1706_03024_gb300 import native as N
from paper_1706_03024_gb300.scene import Scene
from tests.gpu_common import (bin_parity, check_workload as _check_workload,
                              compare_integrated, gpu_batches, integrated_independent,
                              oracle_batches, paired_integrated, require_gpu, totals)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


# ------------------------------------------------------------------------------------------
# Bit-exact integer work


def test_philox_bitwise_against_oracle():
    n = 1_000_000
    rng = np.random.default_rng(11)
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:1000] = 0
    ctr[:1000, 0] = np.arange(1000)
    for seed, med in ((0, 0), (12345, 77), (0xFFFFFFFF, 0xFFFFFFFF)):
        want = oracle.philox(seed, med, ctr)
        c = torch.from_numpy(ctr.view(np.int32)).cuda()
        out = torch.empty_like(c)
        assert N.flr_debug_philox(seed, med, c.data_ptr(), n, out.data_ptr(), 0) == N.FLR_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want)


def test_emission_bins_bitwise_against_oracle():
    sc = sg.cfg2_cornell_box(width=16, height=16, grid=16)
    S = Scene(sc)
    rng = np.random.default_rng(4)
    u = (rng.integers(0, 2 ** 24, size=200_000) / 2.0 ** 24)
    # include every fp32 CDF value itself and its neighbours: the decision boundaries
    edges = []
    for d in range(4):
        f = sc["dyes"]["emit_spec"][d].astype(np.float64)
        cdf = np.cumsum(f) / f.sum()
        for c in cdf.astype(np.float32):
            for k in (-1, 0, 1):
                v = np.float64(c) + k * 2.0 ** -24
                if 0.0 <= v < 1.0:
                    edges.append(np.floor(v * 2 ** 24) / 2 ** 24)
    u = np.concatenate([u, np.array(edges), [0.0, 1 - 2.0 ** -24]]).astype(np.float32)
    ut = torch.from_numpy(u).cuda()
    out = torch.empty(u.shape[0], dtype=torch.int32, device="cuda")
    for d in range(4):
        assert N.flr_debug_sample_emission(S.ctx, d, ut.data_ptr(), u.shape[0], out.data_ptr(),
                                           0) == N.FLR_OK
        torch.cuda.synchronize()
        want = oracle.sample_emission(sc, d, u.astype(np.float64))
        assert np.array_equal(out.cpu().numpy(), want), d


# ------------------------------------------------------------------------------------------
# Statistical parity on the workloads


def test_cfg1_homogeneous_cube_parity():
    sc = sg.cfg1_homogeneous_cube(n_paths=100_000)
    res = _check_workload(sc, 32, 100_000 // 32,
                          forms=("plain", "wavefront", "wavefront_warp", "wavefront_pool"))
    # every launch form traces the same paths: fixed-point tallies bit-identical
    for other in ("wavefront", "wavefront_warp", "wavefront_pool"):
        for a, b in zip(res["plain"], res[other]):
            for key in ("face", "absorbed", "emitted"):
                assert np.array_equal(a[key], b[key]), (other, key)
            assert dict(a["counters"]) == dict(b["counters"]), other
            assert np.allclose(a["film"], b["film"], rtol=1e-5, atol=1e-7 * a["film"].max())


def test_cfg1_analog_and_single_inelastic_parity():
    sc = sg.cfg1_homogeneous_cube(n_paths=64_000)
    _check_workload(sc, 32, 2000, forms=("wavefront",), analog=1)
    _check_workload(sc, 32, 2000, forms=("plain",), max_inelastic=1)


def test_cfg2_cornell_box_reduced_parity():
    sc = sg.cfg2_cornell_box(width=48, height=48, grid=48, n_paths=1)
    _check_workload(sc, 32, 6000, forms=("plain", "wavefront"), path_id_frac=0.97)


def test_cfg2_macro_cell_parity():
    """Local majorants (cells of 4^3 voxels): the oracle walks the same cells in fp64."""
    sc = sg.cfg2_cornell_box(width=48, height=48, grid=48, n_paths=1)
    _check_workload(sc, 32, 6000, forms=("plain", "wavefront"), path_id_frac=0.95, macro_cell=4)


def test_cfg2_empty_space_leap_parity():
    """Leaps out of empty cubes after null collisions (cells of 2^3 voxels); the oracle leaps the
    same way in fp64."""
    sc = sg.cfg2_cornell_box(width=48, height=48, grid=48, n_paths=1)
    _check_workload(sc, 32, 6000, forms=("plain", "wavefront_warp"), path_id_frac=0.95, skip_cell=2)


def test_cfg2_benchmarked_launch_shape_reduced_parity():
    """The launch shape the bench times on the Cornell box (warp-regrouped form, blocks of 128, one
    tracking step per round, empty-space leaps over cells of one voxel) with every criterion: per
    bin of the face, absorbed and emitted tallies, per pixel of the film, same-seed integrated
    tallies within 0.5 %, and an independent seed with the chi-square band on the film."""
    sc = sg.cfg2_cornell_box(width=48, height=48, grid=48, n_paths=1)
    _check_workload(sc, 32, 6000, forms=("wavefront_warp",), path_id_frac=0.95, skip_cell=1,
                    launch={"block_size": 128, "regroup": 1})


def test_cfg2_pool_form_parity_and_equality_with_the_warp_form():
    """The path-pool form (regrouping by event type) on the reduced Cornell box with empty-space
    leaps: the oracle's criteria, and the same fixed-point tallies as the warp form, batch by
    batch."""
    sc = sg.cfg2_cornell_box(width=48, height=48, grid=48, n_paths=1)
    res = _check_workload(sc, 32, 6000, forms=("wavefront_warp", "wavefront_pool"),
                          path_id_frac=0.95, skip_cell=1, launch={"block_size": 128, "regroup": 1})
    for a, b in zip(res["wavefront_warp"], res["wavefront_pool"]):
        for key in ("face", "absorbed", "emitted"):
            assert np.array_equal(a[key], b[key]), key
        assert dict(a["counters"]) == dict(b["counters"])
        assert np.allclose(a["film"], b["film"], rtol=1e-5, atol=1e-7 * a["film"].max())


def test_pool_form_at_full_size_equals_the_warp_form():
    """All 4,194,304 Cornell-box paths: the pool form's fixed-point tallies and per-path event
    counts equal the benchmarked warp form's bit for bit, and the films agree (bit for bit, by the
    fixed-point film sums; test_gpu_film.py asserts that on smaller launches)."""
    sc = sg.cfg2_cornell_box()
    n = sc["params"]["n_paths"]
    S = Scene(sc)
    out = {}
    for form in ("wavefront_warp", "wavefront_pool"):
        pe = torch.zeros(n, dtype=torch.int32, device="cuda")
        f = S.render(form=form, block_size=128, regroup=1, skip_cell=1, path_events=pe).clone()
        out[form] = (S.read(), pe.cpu().numpy(), f)
    a, b = out["wavefront_warp"], out["wavefront_pool"]
    for key in ("face", "absorbed", "emitted"):
        assert np.array_equal(a[0][key], b[0][key]), key
    assert a[0]["counters"] == b[0]["counters"]
    assert np.array_equal(a[1], b[1])
    assert torch.allclose(a[2], b[2], rtol=1e-4, atol=1e-6 * float(a[2].max()))


def test_cfg5_macro_cell_parity():
    sc = sg.cfg5_light_sheet(grid=32, width=32, height=32, n_blobs=40, n_paths=1,
                             sigma_t_ref=20.0)
    _check_workload(sc, 32, 1500, forms=("wavefront",), path_id_frac=0.95, macro_cell=8)


def test_cfg4_blobby_grid_ortho_parity():
    sc = sg.cfg4_adjoint(grid=24, width=24, height=24, n_paths=1)
    _check_workload(sc, 32, 4000, forms=("wavefront",), path_id_frac=0.97)


def test_cfg5_light_sheet_reduced_parity():
    """The light sheet (grids, no solvent mask): the plain and warp forms run the instances that
    take decisions without a grid read where the bounds settle them; the block form does not."""
    sc = sg.cfg5_light_sheet(grid=32, width=32, height=32, n_blobs=40, n_paths=1,
                             sigma_t_ref=20.0)
    _check_workload(sc, 32, 1500, forms=("wavefront", "plain", "wavefront_warp"), path_id_frac=0.95,
                    launch={"block_size": 128, "regroup": 1})


def _minorant_ratio(sc):
    """min over bins of (sigma_s + sigma_a0) / sigma_bar(bin): the library launches the instances
    that skip reads for media with grids, no solvent mask and this ratio >= 0.9."""
    md, dy = sc["medium"], sc["dyes"]
    cmax = md["conc"].reshape(md["conc"].shape[0], -1).max(axis=1).astype(np.float64)
    sig = np.asarray(dy["eps"], np.float64)[:, None] * np.asarray(dy["abs_shape"], np.float64)
    smin = float(md["sigma_s"]) + float(md["sigma_a0"])
    return float((smin / (smin + (sig * cmax[:, None]).sum(axis=0))).min())


@pytest.mark.parametrize("albedo", [0.999, 0.99])
def test_decisions_without_grid_reads_change_nothing(albedo):
    """A medium without a solvent mask, whose sigma_s is most of every bin's majorant, runs the
    kernel instances that skip the grid read when a bound settles the decision (a sure scatter; a
    march whose roulette coin fails against the bound of its estimate). The same medium with an
    all-ones mask has the same coefficients at every point and runs the instances that always
    read: the fixed-point tallies, counters and path events must be identical bit for bit, the
    films agree (their sums are fixed point)."""
    sc = sg.cfg5_light_sheet(grid=48, width=48, height=48, n_blobs=60, n_paths=1, albedo=albedo)
    assert _minorant_ratio(sc) >= 0.9          # the skipping instances are the ones launched
    masked = dict(sc)
    med = dict(sc["medium"])
    nz, ny, nx = med["conc"].shape[1:]
    med["solvent"] = np.ones((nz, ny, nx), dtype=np.uint8)
    masked["medium"] = med
    n = 40_000
    for form, skip in (("plain", 0), ("wavefront_warp", 0), ("wavefront_warp", 1)):
        out = []
        for scene in (sc, masked):
            S = Scene(scene)
            pe = torch.zeros(n, dtype=torch.int32, device="cuda")
            f = S.render(n_paths=n, form=form, path_events=pe, block_size=128, regroup=1,
                         skip_cell=skip)
            out.append((S.read(), f.clone(), pe.cpu().numpy()))
            S.close()
        (a, fa, pa), (b, fb, pb) = out
        for key in ("face", "absorbed", "emitted"):
            assert np.array_equal(a[key], b[key]), (form, key)
        assert dict(a["counters"]) == dict(b["counters"]), form
        assert np.array_equal(pa, pb), form
        assert torch.allclose(fa, fb, rtol=1e-5, atol=1e-7 * float(fa.max())), form
        assert a["counters"]["events"] > 0


def test_cfg3_media_parity_sample():
    media = sg.cfg3_batched_media(n_media=6, seed=0, max_edge=24)
    for m in media[:6]:
        _check_workload(m, 16, 1500, forms=("plain",), path_id_frac=0.97)


def test_uncollided_transmission_gpu_closed_form():
    rng = np.random.default_rng(5)
    n = 6
    conc = rng.uniform(0.0, 2.0, size=(2, n, n, n)).astype(np.float32)
    solvent = (rng.random((n, n, n)) < 0.7).astype(np.uint8)
    dyes = sg.make_dyes([490.0, 500.0], [15.0, 30.0], [620.0, 650.0], [15.0, 15.0],
                        eps=[0.4, 0.3], qy=[0.5, 0.5])
    x, y = 0.41, 0.77
    sc = {"spectrum": sg.spectrum(), "dyes": dyes,
          "medium": sg.grid_medium(conc, solvent, sigma_s=0.8),
          "sources": [sg.pencil_beam((x, y, 1.0), (0, 0, -1), [490.0])],
          "sensor": sg.no_sensor(), "params": sg.params(1_000_000, seed=3)}
    S = Scene(sc)
    S.render(max_events=0)
    r = S.read()
    T = r["face"][:, sg.FACE_NZ, :].sum()
    b = int(math.ceil((490 - sg.LAMBDA0) / sg.DLAMBDA - 0.5))
    tau = oracle.optical_depth(sc, np.array([x, y, 1.0]), np.array([0, 0, -1.0]), 1.0, b)
    exact = math.exp(-tau)
    assert abs(T - exact) <= 3 * math.sqrt(exact * (1 - exact) / 1_000_000), (T, exact)


# ------------------------------------------------------------------------------------------
# Edge cases


def test_empty_ragged_and_single_path_launches():
    sc = sg.cfg1_homogeneous_cube(n_paths=1)
    S = Scene(sc)
    S.render(n_paths=0)
    r = S.read()
    assert r["face"].sum() == 0 and r["counters"]["paths"] == 0
    for n in (1, 31, 257, 1001):
        pe = torch.zeros(n, dtype=torch.int32, device="cuda")
        o = oracle.render(sc, n_paths=n, path_offset=12345, path_events=True)
        for form in ("plain", "wavefront", "wavefront_warp", "wavefront_pool"):
            pe.zero_()
            S.render(n_paths=n, path_offset=12345, form=form, path_events=pe)
            r = S.read()
            assert r["counters"]["paths"] == n
            same = (pe.cpu().numpy().astype(np.uint32) == o["path_events"]).mean()
            assert same >= 0.97, (n, form, same)


def test_ragged_launches_on_a_medium_that_skips_reads():
    """Launches far smaller than the grid of resident warps, on a light-sheet medium whose
    instances take decisions without grid reads: every path traced once, the same paths as the
    oracle."""
    sc = sg.cfg5_light_sheet(grid=32, width=16, height=16, n_blobs=40, n_paths=1, sigma_t_ref=20.0)
    S = Scene(sc)
    for n in (1, 33, 513):
        pe = torch.zeros(n, dtype=torch.int32, device="cuda")
        o = oracle.render(sc, n_paths=n, path_offset=777, path_events=True)
        for form in ("plain", "wavefront_warp"):
            pe.zero_()
            S.render(n_paths=n, path_offset=777, form=form, path_events=pe, block_size=128, regroup=1)
            r = S.read()
            assert r["counters"]["paths"] == n
            assert (pe.cpu().numpy() > 0).all(), (n, form)
            same = (pe.cpu().numpy().astype(np.uint32) == o["path_events"]).mean()
            assert same >= 0.9, (n, form, same)


def test_scattering_only_conserves_exactly_and_empty_medium():
    sc = sg.cfg1_homogeneous_cube(n_paths=50_000)
    sc["dyes"]["eps"] = np.zeros(1, np.float32)
    S = Scene(sc)
    for form in ("plain", "wavefront"):
        S.render(form=form)
        r = S.read()
        assert r["face"].sum() == 1.0
        assert r["counters"]["escapes"] == 50_000
    sc2 = sg.cfg1_homogeneous_cube(n_paths=1000)
    sc2["medium"]["sigma_s"] = 0.0
    sc2["dyes"]["eps"] = np.zeros(1, np.float32)
    S2 = Scene(sc2)
    S2.render()
    r = S2.read()
    assert r["face"][0, sg.FACE_NZ].sum() == 1.0
    assert r["counters"]["events"] == 0


def test_maximum_bins_and_dyes():
    B = 128
    lam0, dl = 380.0, 400.0 / (B - 1)
    lam = lam0 + dl * np.arange(B)
    peaks = [(440, 480), (490, 520), (540, 600), (600, 660)]
    dyes = {"abs_shape": np.stack([np.exp(-0.5 * ((lam - a) / 15) ** 2) for a, _ in peaks]
                                  ).astype(np.float32),
            "emit_spec": np.stack([np.exp(-0.5 * ((lam - e) / 20) ** 2) for _, e in peaks]
                                  ).astype(np.float32),
            "eps": np.array([1.0, 2.0, 1.5, 0.5], np.float32),
            "qy": np.array([0.9, 0.5, 0.7, 0.3], np.float32)}
    sc = {"spectrum": {"lambda0": lam0, "dlambda": dl, "n_bins": B}, "dyes": dyes,
          "medium": sg.homogeneous_medium(4, conc=1.0, sigma_s=10.0),
          "sources": [sg.pencil_beam((0.5, 0.5, 1.0), (0, 0, -1), [440.0, 490.0, 540.0, 600.0])],
          "sensor": sg.ortho_sensor(16, 16, (0, 0, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1)),
          "params": sg.params(1)}
    o = oracle_batches(sc, 16, 2000)
    g = gpu_batches(sc, 16, 2000, form="wavefront")
    for key in ("face", "absorbed", "emitted"):
        assert bin_parity(g, o, key)["ok"], key
        assert compare_integrated(totals(g, key).sum(-1), totals(o, key).sum(-1)) <= 5e-3
    # the warp and pool forms hold the largest tables beside their queues and pools: the same
    # paths, so the same fixed-point tallies as the block form
    for form in ("wavefront_warp", "wavefront_pool"):
        gf = gpu_batches(sc, 16, 2000, form=form)
        for a, b in zip(g, gf):
            for key in ("face", "absorbed", "emitted"):
                assert np.array_equal(a[key], b[key]), (form, key)
    gi = gpu_batches(sc, 16, 2000, form="wavefront", seed=99)
    for key in ("face", "absorbed", "emitted"):
        assert bin_parity(gi, o, key, same_seed=False)["ok"], key
        assert integrated_independent(gi, o, key)[0], key


def test_invalid_arguments_are_rejected():
    sc = sg.cfg1_homogeneous_cube(n_paths=10)
    S = Scene(sc)
    ctx = S.ctx
    a = np.ones((1, 81), np.float32)
    e = np.ones((1, 81), np.float32)
    eps = np.ones(1, np.float32)
    bad_qy = np.array([1.5], np.float32)
    import ctypes as C
    p = lambda arr: arr.ctypes.data_as(C.c_void_p)  # noqa: E731
    assert N.flr_set_dyes(ctx, 1, p(a), p(e), p(eps), p(bad_qy)) == N.FLR_ERR_ARG
    zero_em = np.zeros((1, 81), np.float32)
    assert N.flr_set_dyes(ctx, 1, p(a), p(zero_em), p(eps), p(np.ones(1, np.float32))) == \
        N.FLR_ERR_ARG
    host_grid = np.ones((4, 4, 4), np.float32)
    m = N.flr_medium()
    m.lo[:] = (0, 0, 0)
    m.hi[:] = (1, 1, 1)
    m.dims[:] = (4, 4, 4)
    m.n_dyes = 1
    m.conc[0] = host_grid.ctypes.data
    assert N.flr_set_medium(ctx, m) == N.FLR_ERR_ARG
    assert "device memory" in N.flr_last_error(ctx)
    neg = torch.full((4, 4, 4), -1.0, device="cuda")
    m.conc[0] = neg.data_ptr()
    assert N.flr_set_medium(ctx, m) == N.FLR_ERR_ARG
    m.dims[:] = (4096, 4096, 128)   # 2^31 voxels: rejected before any grid is read
    assert N.flr_set_medium(ctx, m) == N.FLR_ERR_ARG
    assert "2^31" in N.flr_last_error(ctx)
    m.dims[:] = (4, 4, 4)
    par = N.flr_params()
    par.n_paths = 10
    par.max_steps = 100
    par.block_size = 300
    assert N.flr_render(ctx, par, 0) == N.FLR_ERR_ARG
    par.block_size = 0
    par.form = 7
    assert N.flr_render(ctx, par, 0) == N.FLR_ERR_ARG
    par.form = N.FLR_FORM_WAVEFRONT_POOL    # the pool form: one majorant per bin, one wavelength
    par.macro_cell = 4
    assert N.flr_render(ctx, par, 0) == N.FLR_ERR_ARG
    par.macro_cell = 0
    par.hero = 2
    assert N.flr_render(ctx, par, 0) == N.FLR_ERR_ARG
    par.form = N.FLR_FORM_WAVEFRONT_WARP
    par.hero = 5
    assert N.flr_render(ctx, par, 0) == N.FLR_ERR_ARG
    par.hero = 0
    m.conc[0] = host_grid.ctypes.data          # the stream-ordered upload validates the same way
    assert N.flr_set_medium_async(ctx, m, 0) == N.FLR_ERR_ARG
    assert "device memory" in N.flr_last_error(ctx)
    cam = N.flr_sensor()
    cam.kind = N.FLR_SENSOR_PINHOLE
    cam.width = cam.height = 8
    cam.origin[:] = (0.5, 0.5, 0.5)
    cam.U[:] = (1, 0, 0)
    cam.V[:] = (0, 0, 1)
    cam.view[:] = (0, 1, 0)
    cam.fov_y_deg = 40
    assert N.flr_set_sensor(ctx, cam) == N.FLR_OK
    par.form = 0
    assert N.flr_render(ctx, par, 0) == N.FLR_ERR_ARG
    fresh = N.flr_create(0)
    assert N.flr_render(fresh, par, 0) == N.FLR_ERR_STATE
    N.flr_destroy(fresh)
    assert S.status() == N.FLR_OK


def test_step_budget_is_reported_once_by_status():
    """A path cut short at its step budget sets the context's error word: flr_status reports
    FLR_ERR_BUDGET once and then clears it; every launch form reports it."""
    sc = sg.cfg2_cornell_box(width=8, height=8, grid=16, n_paths=2000)
    S = Scene(sc)
    assert S.status() == N.FLR_OK
    for form in ("plain", "wavefront", "wavefront_warp"):
        S.render(form=form, max_steps=1)
        assert S.read()["counters"]["step_budget"] > 0
        assert S.status() == N.FLR_ERR_BUDGET, form
        assert "budget" in N.flr_last_error(S.ctx)
        assert S.status() == N.FLR_OK, form
        S.render(form=form)
        assert S.status() == N.FLR_OK, form


# ------------------------------------------------------------------------------------------
# Full-size workload (the benchmarked configuration): sampled paths and invariants


def _full_size_invariants(c, n, film):
    ends = (c["escapes"] + c["absorbed_dead"] + c["rr_kills"] + c["cap_hits"] + c["step_budget"]
            + c["vf_rejected"])
    assert c["paths"] == n and ends == n
    for name in ("majorant_violations", "nonfinite", "connect_budget", "step_budget"):
        assert c[name] == 0, name
    f = film.double()
    assert torch.isfinite(f).all() and (f >= 0).all() and f.sum() > 0


# the benchmarked launch shape: warp-regrouped form, blocks of 128, one tracking step per round
BENCH_LAUNCH = {"form": "wavefront_warp", "block_size": 128, "regroup": 1}


@pytest.mark.parametrize("launch", [{"form": "wavefront"}, dict(BENCH_LAUNCH, skip_cell=1)],
                         ids=["wavefront", "bench_launch"])
def test_cfg2_full_size_sampled_paths_and_invariants(launch):
    """The Cornell-box workload at full size (512 x 512 pinhole, 16 spp, 128^3 grids, 4,194,304
    paths). Bookkeeping and film checks on every path; event counts of 200 sampled paths against
    the oracle's same paths; and, for the benchmarked launch shape, the integrated tallies of all
    4,194,304 paths against the oracle's same paths (16 batches, same seed) within 0.5 % (rows
    too noisy for that within 4 paired standard errors, see paired_integrated)."""
    sc = sg.cfg2_cornell_box()  # 512 x 512 pinhole, 16 spp, 128^3 grids
    n = sc["params"]["n_paths"]
    assert n == 512 * 512 * 16
    sk = launch.get("skip_cell", 0)
    S = Scene(sc)
    pe = torch.zeros(n, dtype=torch.int32, device="cuda")
    film = S.render(path_events=pe, **launch)
    r = S.read()
    c = r["counters"]
    _full_size_invariants(c, n, film)
    # sampled paths: the oracle traces single paths with the same ids
    rng = np.random.default_rng(2)
    ids = np.sort(rng.choice(n, size=200, replace=False))
    ev = pe.cpu().numpy().astype(np.uint32)
    same = 0
    for pid in ids:
        o = oracle.render(sc, n_paths=1, path_offset=int(pid), film=False, path_events=True,
                          n_threads=1, skip_cell=sk)
        same += int(o["path_events"][0] == ev[pid])
    assert same >= 0.95 * len(ids), same
    # integrated tallies against the oracle's same paths, batch by batch
    K = 16
    m = n // K if launch.get("form") == "wavefront_warp" else 4096
    g = gpu_batches(sc, K, m, film=False, scene_obj=S, skip_cell=sk,
                    **{k: v for k, v in launch.items() if k != "skip_cell"})
    o = oracle_batches(sc, K, m, film=False, skip_cell=sk)
    for key in ("face", "absorbed", "emitted"):
        ok, worst, n_precise, info = paired_integrated(g, o, key)
        assert ok, (key, worst, info)
        if launch.get("form") == "wavefront_warp":
            assert n_precise >= 1, (key, info)


def test_cfg5_light_sheet_full_size_sampled_paths_and_invariants():
    """The light-sheet workload at full size in the benchmarked launch shape: 256^3 x 4 grids
    (larger than the L2), 1024 x 1024 x 81 film, 67,108,864 paths. Bookkeeping and film checks on
    every path; per-path event counts of sampled path ranges against the oracle; integrated
    tallies of the first 262,144 paths against the oracle's same paths (16 batches, same seed)
    within 0.5 % (rows too noisy for that within 4 paired standard errors)."""
    sc = sg.cfg5_light_sheet()
    n = sc["params"]["n_paths"]
    assert n == 1024 * 1024 * 64
    S = Scene(sc)
    pe = torch.zeros(n, dtype=torch.int32, device="cuda")
    launch = dict(BENCH_LAUNCH, skip_cell=0)
    film = S.render(path_events=pe, **launch)
    c = S.read()["counters"]
    _full_size_invariants(c, n, film)
    assert film.shape[-1] == 81 and film.shape[0] * film.shape[1] == 1024 * 1024
    ev = pe.cpu().numpy().astype(np.uint32)
    assert int(ev.astype(np.int64).sum()) == c["events"]
    rng = np.random.default_rng(3)
    starts = np.sort(rng.choice(n // 32, size=8, replace=False)) * 32
    same = total = 0
    for s0 in starts:
        o = oracle.render(sc, n_paths=32, path_offset=int(s0), film=False, path_events=True)
        same += int((o["path_events"] == ev[s0:s0 + 32]).sum())
        total += 32
    assert same >= 0.95 * total, (same, total)
    del pe
    K, m = 16, 16384
    g = gpu_batches(sc, K, m, film=False, scene_obj=S, **launch)
    o = oracle_batches(sc, K, m, film=False)
    for key in ("face", "absorbed", "emitted"):
        ok, worst, n_precise, info = paired_integrated(g, o, key)
        assert ok, (key, worst, info)
