"""The grid lookup every kernel uses (nearest voxel, Sec. 4.1) against the oracle's: the voxel read
bit for bit and sigma_t(x, bin) = s(x)(sigma_s + sigma_a0) + sum_d sig_a[d][bin] c_d(x) to fp32
rounding, on grids with and without a solvent mask, a homogeneous medium, and points outside the
box (clamped to the nearest voxel)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from paper_1706_03024_gb300 import native as N
from paper_1706_03024_gb300.scene import Scene
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu

SCENES = {
    "cornell box (grids and a solvent mask)": lambda: sg.cfg2_cornell_box(width=8, height=8, grid=48,
                                                                          n_paths=1),
    "light sheet (grids, no mask)": lambda: sg.cfg5_light_sheet(grid=40, width=8, height=8, n_blobs=60,
                                                                n_paths=1),
    "adjoint workload (two dyes)": lambda: sg.cfg4_adjoint(grid=24, width=8, height=8, n_paths=1),
    "homogeneous cube": lambda: sg.cfg1_homogeneous_cube(n_paths=1),
}


def _points(sc, rng, n):
    """Points at voxel centres moved by up to 0.4 voxel (away from voxel faces, where an fp32 and
    an fp64 floor may part), and points outside the box along one axis (clamped there)."""
    md = sc["medium"]
    lo, hi = np.asarray(md["lo"], np.float64), np.asarray(md["hi"], np.float64)
    dims = np.asarray(md["dims"] if md.get("dims") is not None else (1, 1, 1), np.int64)   # (nx, ny, nz)
    idx = rng.integers(0, dims, size=(n, 3))
    frac = 0.5 + rng.uniform(-0.4, 0.4, size=(n, 3))
    pts = lo + (idx + frac) * (hi - lo) / dims
    out = pts[: n // 8].copy()
    axis = rng.integers(0, 3, size=out.shape[0])
    side = rng.integers(0, 2, size=out.shape[0])
    for k in range(out.shape[0]):
        a = axis[k]
        out[k, a] = (lo[a] - 0.3 * (hi[a] - lo[a])) if side[k] == 0 else (hi[a] + 0.3 * (hi[a] - lo[a]))
    return np.concatenate([pts, out]).astype(np.float32)


@pytest.mark.parametrize("name", list(SCENES))
def test_grid_lookup_equals_the_oracle(name):
    require_gpu()
    sc = SCENES[name]()
    S = Scene(sc)
    rng = np.random.default_rng(11)
    pts = _points(sc, rng, 20000)
    n = pts.shape[0]
    d_pts = torch.from_numpy(pts).cuda()
    d_sig = torch.empty(n, dtype=torch.float32, device="cuda")
    d_vox = torch.empty(n, dtype=torch.int32, device="cuda")
    B = sc["spectrum"]["n_bins"]
    for b in sorted({0, 10, 22, 28, 44, 60, B - 1}):
        rc = N.flr_debug_sigma_t(S.ctx, d_pts.data_ptr(), n, b, d_sig.data_ptr(), d_vox.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
        assert rc == N.FLR_OK
        torch.cuda.synchronize()
        o_sig, o_vox = oracle.sigma_t_at(sc, pts.astype(np.float64), b)
        g_sig, g_vox = d_sig.cpu().numpy().astype(np.float64), d_vox.cpu().numpy().astype(np.int64)
        assert np.array_equal(g_vox, o_vox), (name, b)
        assert np.allclose(g_sig, o_sig, rtol=4e-6, atol=0.0), (name, b, float(np.abs(g_sig - o_sig).max()))
        assert (o_sig > 0).any() or name.startswith("cornell")
    S.close()


def test_lookup_rejects_bad_arguments():
    require_gpu()
    sc = sg.cfg1_homogeneous_cube(n_paths=1)
    S = Scene(sc)
    d_pts = torch.zeros(3, device="cuda")
    d_sig = torch.zeros(1, device="cuda")
    B = sc["spectrum"]["n_bins"]
    assert N.flr_debug_sigma_t(S.ctx, d_pts.data_ptr(), 1, B, d_sig.data_ptr(), None, 0) == N.FLR_ERR_ARG
    assert N.flr_debug_sigma_t(S.ctx, d_pts.data_ptr(), -1, 0, d_sig.data_ptr(), None, 0) == N.FLR_ERR_ARG
    host = np.zeros(3, np.float32)
    assert N.flr_debug_sigma_t(S.ctx, host.ctypes.data, 1, 0, d_sig.data_ptr(), None, 0) == N.FLR_ERR_ARG
    assert N.flr_debug_sigma_t(S.ctx, d_pts.data_ptr(), 0, 0, d_sig.data_ptr(), None, 0) == N.FLR_OK
    S.close()
