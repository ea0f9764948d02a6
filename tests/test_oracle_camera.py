"""Pins of the oracle's paper-mode light tracer and camera-side estimator (CPU, no GPU).

The paper's own model (Sec. 4.1-4.3) keeps one inelastic event per path, lets the excitation light
reach the dye only uncollided, and renders fluorescence only; its estimator walks from the camera
at the emission wavelength and samples the light at the emission vertex (Eq. 12). The oracle has
both sides of that model: the light tracer with paper_mode=True and render_camera. They are pinned
to a closed form and to each other (two different estimators of one quantity)."""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg
from tests.stats import batch_mean_se, parity_verdict


def slab_scene(W=4, n_paths=1):
    """Uniform collimated beam over the -z face of a non-scattering 1 cm cube of one dye whose
    absorption band overlaps its emission band; orthographic camera on the +z face."""
    dyes = sg.make_dyes([490.0], [30.0], [520.0], [20.0], eps=[2.0], qy=[0.8])
    return {"spectrum": sg.spectrum(), "dyes": dyes, "medium": sg.homogeneous_medium(1, conc=1.0),
            "sources": [sg.rect_source("collimated", (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1),
                                       [490.0])],
            "sensor": sg.ortho_sensor(W, W, (0, 0, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1)),
            "params": sg.params(n_paths, seed=1)}


def slab_closed_form(dyes):
    """Radiance leaving the +z face at bin b: QY p_b / (4 pi) sigma_x * int_0^1
    exp(-sigma_x z) exp(-sigma_b (1 - z)) dz (unit beam power over unit area; p_b the emission pmf
    realised by the fp32 CDF; sigma_x the absorption at the 490 nm line, sigma_b at bin b)."""
    B = sg.N_BINS
    bx = int(math.ceil((490 - sg.LAMBDA0) / sg.DLAMBDA - 0.5))
    sa = dyes["eps"][0].astype(np.float64) * dyes["abs_shape"][0].astype(np.float64)
    sx = float(sa[bx])
    e = dyes["emit_spec"][0].astype(np.float64)
    c32 = (np.cumsum(e) / e.sum()).astype(np.float32)
    c32[-1] = 1.0
    pb = np.diff(np.concatenate([[0.0], c32.astype(np.float64)]))
    out = np.zeros(B)
    for b in range(B):
        sb = float(sa[b])
        f = math.exp(-sb) * math.expm1(sb - sx) / (sb - sx) if abs(sb - sx) > 1e-12 else math.exp(-sx)
        out[b] = float(dyes["qy"][0]) * pb[b] / (4 * math.pi) * sx * f
    return out


def test_slab_closed_form_camera_and_light_paper_mode():
    sc = slab_scene()
    want = slab_closed_form(sc["dyes"])
    K = 8
    cam = [oracle.render_camera(sc, n_paths=16 * 5000, path_offset=k * 16 * 5000)["film"].mean(axis=(0, 1))
           for k in range(K)]
    lt = [oracle.render(sc, n_paths=100_000, path_offset=k * 100_000, paper_mode=True)["film"].mean(axis=(0, 1))
          for k in range(K)]
    for runs in (cam, lt):
        m, se = batch_mean_se(runs)
        big = want > 0.02 * want.max()
        z = (m[big] - want[big]) / se[big]
        assert np.abs(z).max() < 4.5, np.abs(z).max()
        mt, st = batch_mean_se([r.sum() for r in runs])
        assert abs(mt - want.sum()) <= 3.5 * st, (mt, want.sum(), st)


def test_camera_and_light_paper_mode_agree_on_a_scattering_scene():
    """Blobby dyes in a scattering solvent, Lambertian side walls, pinhole camera: the camera-side
    estimator and the paper-mode light tracer estimate the same fluorescence film."""
    sc = sg.paper_mode_scene(n=16, width=8)
    K = 16
    cams = [oracle.render_camera(sc, n_paths=64 * 1000, path_offset=k * 64 * 1000, seed=3)["film"]
            for k in range(K)]
    lts = [oracle.render(sc, n_paths=100_000, path_offset=k * 100_000, paper_mode=True)["film"]
           for k in range(K)]
    a, sa = batch_mean_se([c.sum(axis=(0, 1)) for c in cams])
    b, sb = batch_mean_se([c.sum(axis=(0, 1)) for c in lts])
    v = parity_verdict(a, sa, b, sb, check_chi2=False)
    assert v["ok"], v
    a, sa = batch_mean_se([c.sum(axis=2) for c in cams])
    b, sb = batch_mean_se([c.sum(axis=2) for c in lts])
    v = parity_verdict(a, sa, b, sb, check_chi2=False)
    assert v["ok"], v
    ta, tsa = batch_mean_se([c.sum() for c in cams])
    tb, tsb = batch_mean_se([c.sum() for c in lts])
    assert abs(ta - tb) <= 3 * math.hypot(tsa, tsb), (ta, tb)
    assert ta > 0


def test_paper_mode_rules_are_inert_where_they_do_not_apply():
    """Without scattering, walls or a Lambertian light, the paper's extra rules never fire: paper
    mode equals the one-inelastic-event light tracer path for path."""
    sc = slab_scene()
    a = oracle.render(sc, n_paths=20_000, max_inelastic=1, n_threads=1)
    b = oracle.render(sc, n_paths=20_000, paper_mode=True, n_threads=1)
    assert np.array_equal(a["film"], b["film"])
    assert np.array_equal(a["face"], b["face"])


def test_paper_mode_drops_excitation_scattering():
    """With scattering the full model's film exceeds the paper's (scattered excitation and
    secondary emission add light; Sec. 4.1 drops them)."""
    sc = sg.paper_mode_scene(n=16, width=8)
    full = oracle.render(sc, n_paths=200_000)
    paper = oracle.render(sc, n_paths=200_000, paper_mode=True)
    assert paper["film"].sum() < 0.9 * full["film"].sum()
    assert paper["counters"]["vf_rejected"] > 0


def test_camera_rejects_pencil_beams_and_ragged_path_counts():
    sc = slab_scene()
    with pytest.raises(ValueError):
        oracle.render_camera(sc, n_paths=17)
    sc["sources"] = [sg.pencil_beam((0.5, 0.5, 0.0), (0, 0, 1), [490.0])]
    with pytest.raises(ValueError):
        oracle.render_camera(sc, n_paths=16)
