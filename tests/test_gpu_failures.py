"""Device allocation failures, injected on the host (flr_debug_fail_alloc: the k-th allocation the
library makes fails as out of memory; no device fault is made). Every entry point that allocates
must return an error code, never crash or render from a half-built state, and the library must
work again once allocation succeeds."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import scenegen as sg
from paper_1706_03024_gb300 import native as N
from paper_1706_03024_gb300.scene import Batch, Scene
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def _scene():
    return sg.cfg2_cornell_box(width=16, height=16, grid=24, n_paths=4000)


def _sequence(sc, media):
    """Context creation and upload, a render with empty-space leaps (cell grids), the two-pass
    adjoint (its contribution store), and a batch (its arena and queue): every kind of library
    allocation. Returns the fixed-point tallies of the render and the batch."""
    S = Scene(sc)
    try:
        f = S.render(form="wavefront_warp", block_size=128, regroup=1, skip_cell=1)
        r = S.read()
        adj = torch.ones_like(f)
        D = sc["medium"]["conc"].shape[0]
        gc = torch.zeros((D,) + tuple(sc["medium"]["conc"].shape[1:]), device="cuda")
        gs = torch.zeros(1, device="cuda")
        S.adjoint(adj, gc, gs, form="wavefront_warp", majorant_margin=0.1)
    finally:
        S.close()
    bt = Batch(media, device=0)
    try:
        bt.launch()
        rb = bt.read()
    finally:
        bt.close()
    return r, rb


def test_each_allocation_failing_in_turn_returns_an_error_and_leaves_the_library_usable():
    require_gpu()
    sc = _scene()
    media = sg.cfg3_batched_media(n_media=4, seed=0, max_edge=20, path_scale=0.01)
    want, want_b = _sequence(sc, media)
    failed = 0
    for k in range(1, 40):
        N.flr_debug_fail_alloc(k)
        try:
            _sequence(sc, media)
        except N.FluoroError as e:
            assert e.code in (N.FLR_ERR_OOM, N.FLR_ERR_CUDA), (k, e)
            failed += 1
        finally:
            N.flr_debug_fail_alloc(0)
        torch.cuda.synchronize()
    assert failed >= 10                       # the sequence allocates at least this many buffers
    got, got_b = _sequence(sc, media)         # everything works again, with the same results
    for key in ("face", "absorbed", "emitted"):
        assert np.array_equal(got[key], want[key]), key
        assert np.array_equal(got_b[key], want_b[key]), key


def test_a_failed_grid_upload_leaves_no_medium_to_render():
    """The packed grid is re-allocated for a larger medium; when that fails the previous grid is
    already gone, so the context refuses to render (FLR_ERR_STATE) until an upload succeeds."""
    require_gpu()
    small = sg.cfg2_cornell_box(width=16, height=16, grid=16, n_paths=2000)
    large = sg.cfg2_cornell_box(width=16, height=16, grid=32, n_paths=2000)
    S = Scene(small)
    S.render()
    N.flr_debug_fail_alloc(1)
    try:
        with pytest.raises(N.FluoroError) as e:
            S.set_medium(large["medium"])
        assert e.value.code == N.FLR_ERR_OOM
    finally:
        N.flr_debug_fail_alloc(0)
    with pytest.raises(N.FluoroError) as e:
        S.render()
    assert e.value.code == N.FLR_ERR_STATE
    S.set_medium(large["medium"])
    S.render()
    assert S.read()["counters"]["paths"] == 2000
    S.close()


def test_hook_rejects_negative_counts():
    require_gpu()
    assert N.flr_debug_fail_alloc(-1) == N.FLR_ERR_ARG
    assert N.flr_debug_fail_alloc(0) == N.FLR_OK
