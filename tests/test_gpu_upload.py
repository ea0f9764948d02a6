"""The medium upload ordered on a stream (flr_set_medium_async) against the device-synchronising
one (flr_set_medium): the same packed grid, maxima and majorants, so the same render bit for bit
on the fixed-point tallies; and the same validation."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import scenegen as sg
from paper_1706_03024_gb300.scene import Scene
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scene", ["cornell", "sheet"])
def test_stream_ordered_upload_renders_the_same(scene):
    require_gpu()
    sc = (sg.cfg2_cornell_box(width=32, height=32, grid=32, n_paths=20000) if scene == "cornell"
          else sg.cfg5_light_sheet(grid=32, width=32, height=32, n_blobs=40, n_paths=20000,
                                   sigma_t_ref=20.0))
    md = sc["medium"]
    conc = torch.from_numpy(np.ascontiguousarray(md["conc"])).cuda()
    grids = {"conc": conc}
    if md.get("solvent") is not None:
        grids["solvent"] = torch.from_numpy(np.ascontiguousarray(md["solvent"])).cuda()
    torch.cuda.synchronize()
    A, B = Scene(sc), Scene(sc)
    st = torch.cuda.Stream()
    A.set_medium(md, grids=grids)
    B.set_medium(md, grids=grids, stream=st)
    fa = A.render(form="wavefront_warp", block_size=128, regroup=1, skip_cell=1).clone()
    ra = A.read()
    fb = B.render(form="wavefront_warp", block_size=128, regroup=1, skip_cell=1, stream=st)
    rb = B.read(stream=st)
    fb = fb.clone()
    for key in ("face", "absorbed", "emitted"):
        assert np.array_equal(ra[key], rb[key]), key
    assert dict(ra["counters"]) == dict(rb["counters"])
    assert torch.allclose(fa, fb, rtol=1e-5, atol=1e-7 * float(fa.max()))
    A.close()
    B.close()


def test_stream_ordered_upload_rejects_negative_concentrations():
    require_gpu()
    sc = sg.cfg4_adjoint(grid=16, width=8, height=8, n_paths=100)
    md = sc["medium"]
    conc = torch.from_numpy(np.ascontiguousarray(md["conc"])).cuda()
    conc[0, 3, 4, 5] = -1.0
    S = Scene(sc)
    st = torch.cuda.Stream()
    with pytest.raises(Exception, match="negative"):
        S.set_medium(md, grids={"conc": conc}, stream=st)
    with pytest.raises(Exception, match="negative"):
        S.set_medium(md, grids={"conc": conc})
    S.close()
