"""The index-checked build (libfluoro_checked.so, FLR_CHECKED): every launch form on small versions
of the workloads, with every device index tested before its access, leaves no violation; and a
violation provoked by the debug entry is reported by flr_status as FLR_ERR_CHECK (the access is
skipped, nothing traps). Runs in a child process: the binding loads one library per process."""
import os
import subprocess
import sys

import pytest

from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run_all():
    import torch

    import scenegen as sg
    from paper_1706_03024_gb300 import native as N
    from paper_1706_03024_gb300.scene import Batch, Scene

    assert N.flr_checked_build() == 1
    cases = [
        (sg.cfg1_homogeneous_cube(n_paths=20000), [{"form": f} for f in ("plain", "wavefront", "wavefront_warp")]),
        (sg.cfg2_cornell_box(width=32, height=32, grid=32, n_paths=40000),
         [{"form": "plain"}, {"form": "wavefront"}, {"form": "wavefront_warp"},
          {"form": "wavefront_warp", "skip_cell": 2}, {"form": "wavefront_warp", "macro_cell": 4},
          {"form": "plain", "macro_cell": 4}, {"form": "plain", "hero": 4, "skip_cell": 1},
          {"form": "wavefront_warp", "hero": 4, "skip_cell": 1},
          {"form": "wavefront_warp", "paper_mode": True}, {"form": "wavefront_pool", "skip_cell": 1}]),
        # grids without a solvent mask: the instances that skip reads a bound settles
        (sg.cfg5_light_sheet(grid=32, width=32, height=32, n_blobs=40, n_paths=20000,
                             sigma_t_ref=20.0),
         [{"form": "wavefront_warp"}, {"form": "plain"}, {"form": "wavefront_warp", "skip_cell": 1}]),
        # dielectric faces and glossy walls
        (sg.vial_scene(conc_gpl=1.0, ior=1.33, width=24, height=24, n_paths=20000, grid=32),
         [{"form": f} for f in ("plain", "wavefront", "wavefront_warp", "wavefront_pool")]),
        (sg.cfg2_cornell_box(width=32, height=32, grid=32, n_paths=20000, wall_gloss=0.5,
                             wall_exponent=20.0),
         [{"form": "wavefront_warp", "skip_cell": 1}, {"form": "plain"}]),
    ]
    for sc, launches in cases:
        S = Scene(sc)
        for kw in launches:
            S.render(**kw)
            assert S.status() == N.FLR_OK, (sc.get("name"), kw, N.flr_last_error(S.ctx))
        S.close()
    # the camera-side estimator, both forms
    sc = sg.paper_mode_scene(n=16, width=16, spp=64)
    S = Scene(sc)
    for form in ("plain", "wavefront_warp"):
        S.render_camera(n_paths=16 * 16 * 64, form=form)
        assert S.status() == N.FLR_OK, form
    S.close()
    # the adjoint, both forms
    sc = sg.cfg4_adjoint(grid=16, width=16, height=16, n_paths=20000)
    S = Scene(sc)
    film = S.render(form="wavefront_warp", majorant_margin=0.1)
    adj = (2.0 * film).contiguous()
    gc = torch.zeros(S.conc_t.shape, dtype=torch.float32, device="cuda")
    gs = torch.zeros(1, dtype=torch.float32, device="cuda")
    for form in ("plain", "wavefront_warp"):
        S.adjoint(adj, gc, gs, majorant_margin=0.1, form=form)
        assert S.status() == N.FLR_OK, form
    # the batched form
    bt = Batch(sg.cfg3_batched_media(n_media=8, seed=0, max_edge=24, path_scale=0.05), device=0)
    bt.launch()
    bt.read()
    bt.close()
    assert S.status() == N.FLR_OK
    # a provoked violation is reported, once
    assert N.flr_debug_check(7, 100) == N.FLR_OK
    assert S.status() == N.FLR_OK
    assert N.flr_debug_check(123, 100) == N.FLR_OK
    rc = S.status()
    assert rc == N.FLR_ERR_CHECK, rc
    assert "index 123" in N.flr_last_error(S.ctx)
    assert S.status() == N.FLR_OK
    S.close()
    print("checked build: clean")


def test_checked_build_runs_every_form_without_violations():
    require_gpu()
    from paper_1706_03024_gb300 import build as B
    B.build(checked=True)
    env = dict(os.environ, FLR_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", "import tests.test_gpu_checked as t; t._run_all()"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build: clean" in r.stdout
