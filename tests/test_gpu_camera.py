"""The paper's single-inelastic model on the GPU: the light tracer's paper mode and the camera-side
estimator (flr_render_camera), against the oracle's, a closed form, and each other.

The paper's own estimator (Sec. 4.1-4.3, Eq. 12) walks from the camera at the emission wavelength
and samples the light at every collision; the light tracer in paper mode estimates the same
fluorescence film from the light side. The GPU estimates the transmittances by ratio tracking, the
oracle evaluates them exactly, so the comparisons are statistical."""
import math

import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from paper_1706_03024_gb300.native import FluoroError
from paper_1706_03024_gb300.scene import Scene
from tests.gpu_common import require_gpu
from tests.stats import batch_mean_se, parity_verdict
from tests.test_gpu_parity import _check_workload
from tests.test_oracle_camera import slab_closed_form, slab_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def gpu_camera(S, K, n_per, seed=None, form="wavefront_warp"):
    return [S.render_camera(n_paths=n_per, path_offset=k * n_per, seed=seed, form=form)
            .double().cpu().numpy() for k in range(K)]


def test_slab_closed_form_gpu_camera_and_light_paper_mode():
    sc = slab_scene()
    want = slab_closed_form(sc["dyes"])
    S = Scene(sc)
    K = 16
    cam = [f.mean(axis=(0, 1)) for f in gpu_camera(S, K, 16 * 20_000)]
    # independent path ranges, alternating the plain and the warp-regrouped forms
    lt = [S.render(n_paths=200_000, path_offset=k * 200_000, form=("plain", "wavefront_warp")[k % 2],
                   paper_mode=True).double().cpu().numpy().mean(axis=(0, 1)) for k in range(K)]
    for runs in (cam, lt):
        m, se = batch_mean_se(runs)
        big = want > 0.02 * want.max()
        z = (m[big] - want[big]) / se[big]
        assert np.abs(z).max() < 4.5, np.abs(z).max()
        mt, st = batch_mean_se([r.sum() for r in runs])
        assert abs(mt - want.sum()) <= 3.5 * st + 2e-3 * want.sum(), (mt, want.sum(), st)


def test_camera_forms_agree():
    """The plain and the warp-regrouped camera forms draw the same random numbers for the same
    paths: the same film (fixed-point sums)."""
    sc = sg.paper_mode_scene(n=32, width=16)
    S = Scene(sc)
    n = 256 * 500
    a = S.render_camera(n_paths=n, seed=4, form="plain").double().cpu().numpy()
    b = S.render_camera(n_paths=n, seed=4, form="wavefront_warp").double().cpu().numpy()
    assert np.allclose(a, b, rtol=1e-4, atol=1e-6 * np.abs(a).max())
    assert a.sum() > 0


@pytest.mark.parametrize("form", ["plain", "wavefront_warp"])
def test_gpu_camera_matches_oracle_camera(form):
    sc = sg.paper_mode_scene(n=16, width=8)
    S = Scene(sc)
    K, n = 16, 64 * 1000
    g = gpu_camera(S, K, n, seed=3, form=form)
    o = [oracle.render_camera(sc, n_paths=n, path_offset=k * n, seed=3)["film"] for k in range(K)]
    for axis in ((0, 1), 2):
        a, sa = batch_mean_se([x.sum(axis=axis) for x in g])
        b, sb = batch_mean_se([x.sum(axis=axis) for x in o])
        v = parity_verdict(a, sa, b, sb, check_chi2=False)
        assert v["ok"], (axis, v)
    ta, tsa = batch_mean_se([x.sum() for x in g])
    tb, tsb = batch_mean_se([x.sum() for x in o])
    assert abs(ta - tb) <= 3 * math.hypot(tsa, tsb) + 5e-3 * tb, (ta, tb)
    c = S.read()["counters"]
    assert c["majorant_violations"] == 0 and c["step_budget"] == 0 and c["connections"] > 0


def test_gpu_light_paper_mode_parity_and_forms():
    """Paper mode on the light side: oracle parity for the plain and warp-regrouped forms, which
    trace the same paths (bit-identical fixed-point tallies)."""
    sc = sg.paper_mode_scene(n=16, width=8)
    res = _check_workload(sc, 32, 4000, forms=("plain", "wavefront_warp"), paper_mode=True)
    for a, b in zip(res["plain"], res["wavefront_warp"]):
        for key in ("face", "absorbed", "emitted"):
            assert np.array_equal(a[key], b[key]), key
        assert a["counters"]["vf_rejected"] == b["counters"]["vf_rejected"] > 0


def test_gpu_camera_and_light_paper_mode_agree():
    """Two estimators of one film, both on the GPU, on a 32^3 grid and a 16x16 film."""
    sc = sg.paper_mode_scene(n=32, width=16)
    S = Scene(sc)
    K = 16
    cams = gpu_camera(S, K, 256 * 2000, seed=5)
    lts = [S.render(n_paths=400_000, path_offset=k * 400_000, form="wavefront_warp",
                    paper_mode=True).double().cpu().numpy() for k in range(K)]
    for axis in ((0, 1), 2):
        a, sa = batch_mean_se([x.sum(axis=axis) for x in cams])
        b, sb = batch_mean_se([x.sum(axis=axis) for x in lts])
        v = parity_verdict(a, sa, b, sb, check_chi2=False)
        assert v["ok"], (axis, v)
    ta, tsa = batch_mean_se([x.sum() for x in cams])
    tb, tsb = batch_mean_se([x.sum() for x in lts])
    assert abs(ta - tb) <= 3 * math.hypot(tsa, tsb), (ta, tb, tsa, tsb)


def test_camera_rejects_bad_arguments():
    sc = slab_scene()
    S = Scene(sc)
    with pytest.raises(FluoroError):
        S.render_camera(n_paths=17)                 # not a multiple of the pixel count
    with pytest.raises(FluoroError):
        S.render_camera(n_paths=16, path_offset=5)
    sc2 = slab_scene()
    sc2["sources"] = [sg.pencil_beam((0.5, 0.5, 0.0), (0, 0, 1), [490.0])]
    with pytest.raises(FluoroError):
        Scene(sc2).render_camera(n_paths=16)        # a pencil beam has no fluence density
    f = S.render_camera(n_paths=0)
    assert float(f.abs().sum()) == 0.0


def test_camera_full_size_invariants():
    """A 64^3 grid, 256x256 film, 8 paths per pixel: finite, non-negative, deterministic for a
    fixed seed (the film's sums are fixed point), and its total within 5 % of the paper-mode light
    tracer's at the same size (the two estimators' batch errors are both below 1 % here)."""
    sc = sg.paper_mode_scene(n=64, width=256)
    S = Scene(sc)
    n = 256 * 256 * 8
    f1 = S.render_camera(n_paths=n, seed=9).clone()
    f2 = S.render_camera(n_paths=n, seed=9).clone()
    assert torch.isfinite(f1).all() and (f1 >= 0).all()
    assert torch.allclose(f1, f2, rtol=1e-4, atol=1e-6 * float(f1.max()))
    lt = S.render(n_paths=8_000_000, form="wavefront_warp", paper_mode=True).clone()
    a, b = float(f1.double().sum()), float(lt.double().sum())
    assert abs(a - b) <= 0.05 * b, (a, b)
