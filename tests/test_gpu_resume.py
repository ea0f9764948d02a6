"""Checkpoint and resume of a render. The tallies are additive and every random number is a
function of (seed, medium, path id, step, slot), so a render split at any path id and resumed with
accumulation gives the uninterrupted render's fixed-point tallies bit for bit, and its film up to one
fp32 rounding per launch (each launch folds its exact sums into the fp32 film); a checkpoint is (tallies, film, next path id)."""
import numpy as np
import pytest

import scenegen as sg
from paper_1706_03024_gb300.scene import Scene
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("form", ["plain", "wavefront_warp"])
def test_split_and_resumed_render_equals_the_whole(form):
    sc = sg.cfg2_cornell_box(width=32, height=32, grid=32, n_paths=1)
    S = Scene(sc)
    n, cut = 60_000, 23_457
    whole = S.render(n_paths=n, form=form).double().cpu().numpy()
    r_whole = S.read()
    # a split render: the first part, then the rest resumed from the next path id
    a = S.render(n_paths=cut, form=form).double().cpu().numpy()
    b = S.render(n_paths=n - cut, path_offset=cut, form=form, accumulate=True).double().cpu().numpy()
    r_split = S.read()
    for key in ("face", "absorbed", "emitted"):
        assert np.array_equal(r_whole[key], r_split[key]), key
    assert r_whole["counters"] == r_split["counters"]
    # each call scales its film contributions by 1 / (its own path count), and the accumulated
    # film holds both calls (b = a + the rest's film): undo the per-call scales
    merged = a * cut / n + (b - a) * (n - cut) / n
    scale = np.abs(whole).max()
    assert np.allclose(merged, whole, rtol=1e-4, atol=1e-6 * scale)
