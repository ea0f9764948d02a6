"""The film's fixed-point sums: each contribution (Eq. 3-6) is added as a 64-bit integer in units of
2^-32, and the launch's sums are folded into the fp32 film when it ends.

- The sums do not depend on the order of the additions: the film is the same bit for bit whatever
  the launch shape (block size, regroup depth) and from one launch to the next.
- Forms that trace the same paths with the same connection arithmetic give the same film bit for
  bit (as their fixed-point tallies are): the plain, warp and pool forms, also in the instances
  that skip grid reads; the plain and warp hero forms; the camera-side estimator's two forms.
- accumulate = 1 adds the launch's film to the previous one with one fp32 addition per value, and
  a launch without paths clears the film.
- At 1e8 paths of the homogeneous cube (a pencil beam seen along its axis puts about a sixth of
  all contributions on one film value) the film's sum and its brightest value agree with the
  oracle's fp64 estimate; fp32 atomics lost 10 % of the sum and 62 % of that value there.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from paper_1706_03024_gb300.scene import Scene
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _diff(a, b):
    d = (a != b)
    n = int(d.sum())
    if n == 0:
        return "equal"
    rel = float(((a - b).abs() / b.abs().clamp_min(1e-30))[d].max())
    return f"{n} of {a.numel()} values differ, max relative difference {rel:.3g}"


def _cornell():
    return sg.cfg2_cornell_box(width=64, height=64, grid=48, n_paths=60_000)


def _sheet():
    return sg.cfg5_light_sheet(grid=48, width=48, height=48, n_blobs=60, n_paths=40_000, albedo=0.999)


def test_the_film_does_not_depend_on_the_launch_shape():
    S = Scene(_cornell())
    try:
        ref = S.render(form="wavefront_warp", block_size=128, regroup=1).clone()
        assert float(ref.sum()) > 0.0
        for kw in ({"form": "wavefront_warp", "block_size": 128, "regroup": 1},
                   {"form": "wavefront_warp", "block_size": 64, "regroup": 1},
                   {"form": "wavefront_warp", "block_size": 256, "regroup": 2},
                   {"form": "wavefront_warp", "block_size": 128, "regroup": 4}):
            f = S.render(**kw)
            assert torch.equal(f, ref), (kw, _diff(f, ref))
        p = S.render(form="plain", block_size=128).clone()
        for b in (64, 256):
            f = S.render(form="plain", block_size=b)
            assert torch.equal(f, p), (b, _diff(f, p))
    finally:
        S.close()


@pytest.mark.parametrize("scene", ["cornell box", "light sheet"])
def test_forms_that_trace_the_same_connections_give_the_same_film(scene):
    """The plain, warp and pool forms trace the same paths, and their connections draw the same
    uniforms into the same arithmetic (the light sheet: in the instances that skip grid reads)."""
    sc = _cornell() if scene == "cornell box" else _sheet()
    forms = ("wavefront_warp", "wavefront_pool", "plain") if scene == "cornell box" else ("wavefront_warp", "plain")
    S = Scene(sc)
    try:
        films = {f: S.render(form=f, block_size=128, regroup=1, skip_cell=1).clone() for f in forms}
    finally:
        S.close()
    w = films["wavefront_warp"]
    assert float(w.sum()) > 0.0
    for f in forms[1:]:
        assert torch.equal(films[f], w), (f, _diff(films[f], w))


def test_hero_forms_give_the_same_film():
    S = Scene(_cornell())
    try:
        a = S.render(form="plain", hero=4).clone()
        b = S.render(form="wavefront_warp", block_size=128, regroup=1, hero=4).clone()
    finally:
        S.close()
    assert float(a.sum()) > 0.0
    assert torch.equal(a, b), _diff(b, a)


def test_camera_forms_give_the_same_film():
    sc = sg.paper_mode_scene(n=16, width=32)
    S = Scene(sc)
    try:
        n = 32 * 32 * 8
        a = S.render_camera(n_paths=n, form="plain").clone()
        b = S.render_camera(n_paths=n, form="wavefront_warp").clone()
    finally:
        S.close()
    assert float(a.sum()) > 0.0
    assert torch.equal(a, b), _diff(b, a)


def test_accumulate_adds_the_launch_film_once_per_value():
    S = Scene(_cornell())
    try:
        kw = {"form": "wavefront_warp", "block_size": 128, "regroup": 1, "n_paths": 20_000}
        a = S.render(path_offset=0, **kw).clone()
        b = S.render(path_offset=20_000, **kw).clone()
        S.render(path_offset=0, **kw)
        both = S.render(path_offset=20_000, accumulate=True, **kw).clone()
        assert torch.equal(both, a + b)
        S.render(n_paths=0, form="wavefront_warp")     # a launch without paths clears the film
        assert float(S.film.abs().sum()) == 0.0
    finally:
        S.close()


def test_full_size_cube_film_keeps_every_contribution():
    """1e8 paths of the homogeneous cube: the GPU film's sum and its brightest value (the beam's
    entry pixel at the excitation bin) against the oracle's fp64 batch means over 16 batches of
    250,000 other path ids (the GPU's own Monte Carlo error is 5x smaller): within 4 combined
    standard errors."""
    n = 100_000_000
    sc = sg.cfg1_homogeneous_cube(n_paths=n)
    S = Scene(sc)
    try:
        g = S.render(form="wavefront_warp", block_size=128, regroup=1).double().cpu().numpy()
    finally:
        S.close()
    hot = np.unravel_index(int(np.argmax(g)), g.shape)
    assert hot[:2] == (32, 32)                # the beam's axis is the film's centre
    K, m = 16, 250_000
    sums, hots = [], []
    for k in range(K):
        r = oracle.render(sc, n_paths=m, path_offset=n + k * m)
        sums.append(float(r["film"].sum()))
        hots.append(float(r["film"][hot]))
    for name, got, vals in (("film sum", float(g.sum()), sums), ("brightest value", float(g[hot]), hots)):
        mean = float(np.mean(vals))
        se_o = float(np.std(vals, ddof=1) / np.sqrt(K))
        se = float(np.hypot(se_o, se_o * np.sqrt(K * m / n)))
        assert abs(got - mean) <= 4.0 * se, (name, got, mean, se)
