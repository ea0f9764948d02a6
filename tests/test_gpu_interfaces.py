"""Dielectric faces and glossy walls on the GPU (the glass vials and the glossy Cornell box of the
paper's Sec. 5) against the oracle, whose physics tests/test_oracle_interfaces.py pins: per-bin and
per-pixel parity on a vial of dye solution and on a glossy Cornell box, every launch form tracing
the same paths (bit-identical fixed-point tallies), closed forms on the GPU itself (the
normal-incidence slab series, the head-on film of a glossy floor), and the settings that are not
modelled rejected."""
import math

import numpy as np
import pytest
import torch

import scenegen as sg
from paper_1706_03024_gb300 import native as N
from paper_1706_03024_gb300.scene import Batch, Scene
from tests.gpu_common import check_workload, require_gpu
from tests.stats import binomial_se

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_vial_parity_and_forms_agree():
    """A 1 cm cuvette of scattering dye solution (index 1.33) lit through its -x face, seen
    head-on through its front face."""
    sc = sg.vial_scene(conc_gpl=1.0, ior=1.33, width=24, height=24, n_paths=1)
    res = check_workload(sc, 32, 4000, forms=("plain", "wavefront", "wavefront_warp",
                                              "wavefront_pool"), path_id_frac=0.97)
    for other in ("wavefront", "wavefront_warp", "wavefront_pool"):
        for a, b in zip(res["plain"], res[other]):
            for key in ("face", "absorbed", "emitted"):
                assert np.array_equal(a[key], b[key]), (other, key)
            assert dict(a["counters"]) == dict(b["counters"]), other
    c = res["plain"][0]["counters"]
    assert c["iface_reflections"] > 0 and c["majorant_violations"] == 0


def test_vial_with_a_voxelised_vial_and_leaps():
    """The dye in a cylinder on a 32^3 grid with empty-space leaps, in the benchmarked launch shape."""
    sc = sg.vial_scene(conc_gpl=2.0, ior=1.5, width=24, height=24, n_paths=1, grid=32)
    check_workload(sc, 32, 3000, forms=("wavefront_warp",), path_id_frac=0.95, skip_cell=1,
                   launch={"block_size": 128, "regroup": 1})


def test_glossy_cornell_box_parity():
    sc = sg.cfg2_cornell_box(width=48, height=48, grid=48, n_paths=1, wall_gloss=0.5,
                             wall_exponent=20.0)
    res = check_workload(sc, 32, 6000, forms=("plain", "wavefront_warp", "wavefront_pool"),
                         path_id_frac=0.95, skip_cell=1)
    for other in ("wavefront_warp", "wavefront_pool"):
        for a, b in zip(res["plain"], res[other]):
            for key in ("face", "absorbed", "emitted"):
                assert np.array_equal(a[key], b[key]), (other, key)


def test_slab_series_on_the_gpu():
    n, tau, N_ = 1.5, 1.0, 1_000_000
    dyes = sg.make_dyes([490.0], [15.0], [650.0], [15.0], eps=[0.0], qy=[0.0])
    med = sg.homogeneous_medium(1, conc=1.0, sigma_a0=tau)
    med["ior"] = n
    sc = {"spectrum": sg.spectrum(), "dyes": dyes, "medium": med,
          "sources": [sg.pencil_beam((0.5, 0.5, 1.0), (0, 0, -1), [490.0])],
          "sensor": sg.no_sensor(), "params": sg.params(N_)}
    S = Scene(sc)
    for form in ("plain", "wavefront_warp", "wavefront_pool"):
        S.render(form=form, film=False)
        r = S.read()
        F0 = ((n - 1) / (n + 1)) ** 2
        e1, e2 = math.exp(-tau), math.exp(-2 * tau)
        T = (1 - F0) ** 2 * e1 / (1 - F0 ** 2 * e2)
        R = F0 + (1 - F0) ** 2 * F0 * e2 / (1 - F0 ** 2 * e2)
        assert abs(r["face"][0, sg.FACE_NZ].sum() - T) <= 4 * binomial_se(T, N_), form
        assert abs(r["face"][0, sg.FACE_PZ].sum() - R) <= 4 * binomial_se(R, N_), form


def test_glossy_floor_film_head_on_on_the_gpu():
    rho, g, e, th = 0.8, 0.6, 20.0, math.radians(25.0)
    med = sg.homogeneous_medium(1, conc=0.0, wall_mask=1 << sg.FACE_NZ, wall_albedo=rho)
    med["wall_gloss"], med["wall_exponent"] = g, e
    z0 = 0.25
    d = (math.sin(th), 0.0, -math.cos(th))
    cam = sg.ortho_sensor(8, 8, (0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0))
    sc = {"spectrum": sg.spectrum(), "dyes": sg.make_dyes([490.0], [15.0], [650.0], [15.0],
                                                          eps=[0.0], qy=[0.0]),
          "medium": med, "sources": [sg.pencil_beam((0.5 - z0 * math.tan(th), 0.5, z0), d, [490.0])],
          "sensor": cam, "params": sg.params(4096)}
    S = Scene(sc)
    for form in ("plain", "wavefront_warp", "wavefront_pool"):
        film = S.render(form=form).double().cpu().numpy()
        want = rho * ((1 - g) / math.pi + g * (e + 2) / (2 * math.pi) * math.cos(th) ** e) * 64
        assert film[4, 4].sum() == pytest.approx(want, rel=2e-4), form
        film[4, 4] = 0.0
        assert film.sum() == 0.0


def test_settings_that_are_not_modelled_are_rejected():
    sc = sg.vial_scene(width=8, height=8, n_paths=100)
    sc["sensor"] = sg.pinhole_sensor(8, 8, eye=(0.5, -2.0, 0.5), right=(1, 0, 0), up=(0, 0, 1),
                                     forward=(0, 1, 0), fov_y_deg=30.0)
    S = Scene(sc)
    with pytest.raises(RuntimeError):
        S.render()
    S.render(film=False)   # without a film the sensor does not matter
    sc2 = sg.vial_scene(width=8, height=8, n_paths=100)
    S2 = Scene(sc2)
    S2.render()
    for kw in ({"hero": 2}, {"paper_mode": True}):
        with pytest.raises(RuntimeError):
            S2.render(**kw)
    with pytest.raises(RuntimeError):
        S2.render_camera(n_paths=64)
    glossy = sg.cfg3_batched_media(n_media=2, seed=0, max_edge=16)
    glossy[1]["medium"]["wall_gloss"] = 0.5
    with pytest.raises(RuntimeError):
        Batch(glossy)
