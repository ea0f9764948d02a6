"""flr_render_noalloc: the single-scene render for callers that cannot allocate device memory.

Some callers may not call cudaMalloc at all: their device memory belongs to another allocator (a
framework's caching pool that has reserved the GPU), or they run under a fixed memory budget that
forbids allocation at run time. This entry point keeps all of its scratch in one static device
array instead. Here it must give what the allocating entry points give (flr_render followed by
flr_read_tallies) on the same paths: the same fixed-point tallies, bit for bit, and the same film
up to fp32 rounding (this entry point adds contributions by fp32 atomics, flr_render sums them in
fixed point) -- on two calls in a row, since every call reuses the array -- in
every launch form, with and without grids. Settings it cannot honour are rejected, and a path cut
short at its step budget is reported.
This file is collected last so that a stop-at-first-failure run has already run everything else.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import scenegen as sg
from paper_1706_03024_gb300 import native as N
from paper_1706_03024_gb300.scene import Scene, make_sensor, make_source
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu

_FORMS = {"plain": N.FLR_FORM_PLAIN, "wavefront": N.FLR_FORM_WAVEFRONT,
          "wavefront_warp": N.FLR_FORM_WAVEFRONT_WARP}


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _noalloc(sc, conc_t, solv_t, n_paths, form, film, **over):
    dy, md, sp = sc["dyes"], sc["medium"], sc["spectrum"]
    D = int(dy["eps"].shape[0])
    m = N.flr_medium()
    m.lo[:] = md["lo"]
    m.hi[:] = md["hi"]
    m.n_dyes = D
    for d in range(D):
        m.dye_ids[d] = d
        if conc_t is not None:
            m.conc[d] = conc_t[d].data_ptr()
        else:
            m.conc_uniform[d] = float(md["conc_uniform"][d])
    if conc_t is not None:
        _, nz, ny, nx = conc_t.shape
        m.dims[:] = (nx, ny, nz)
    m.solvent = solv_t.data_ptr() if solv_t is not None else None
    m.sigma_s = md["sigma_s"]
    m.sigma_a0 = md["sigma_a0"]
    m.wall_mask = md["wall_mask"]
    m.wall_albedo = md["wall_albedo"]
    m.ior = md.get("ior", 1.0)
    m.wall_gloss = md.get("wall_gloss", 0.0)
    m.wall_exponent = md.get("wall_exponent", 0.0)
    srcs = (N.flr_source * len(sc["sources"]))(*[make_source(s) for s in sc["sources"]])
    p = N.flr_params()
    p.n_paths = n_paths
    p.seed = sc["params"]["seed"]
    p.n_rr = sc["params"]["n_rr"]
    p.max_inelastic = -1
    p.form = _FORMS[form]
    p.max_events = sc["params"]["max_events"]
    p.max_steps = sc["params"]["max_steps"]
    p.film = film.data_ptr()
    for k, v in over.items():
        setattr(p, k, v)
    B = sp["n_bins"]
    face, absorbed = np.zeros((2, 6, B)), np.zeros((D + 1, B))
    emitted, counters = np.zeros((D, B)), np.zeros(N.FLR_NCOUNTERS, np.uint64)
    a = np.ascontiguousarray(dy["abs_shape"], np.float32)
    e = np.ascontiguousarray(dy["emit_spec"], np.float32)
    eps = np.ascontiguousarray(dy["eps"], np.float32)
    qy = np.ascontiguousarray(dy["qy"], np.float32)
    rc = N.flr_render_noalloc(sp["lambda0"], sp["dlambda"], B, D, _ptr(a), _ptr(e), _ptr(eps),
                              _ptr(qy), m, len(sc["sources"]), srcs, make_sensor(sc["sensor"]), p,
                              _ptr(face), _ptr(absorbed), _ptr(emitted), _ptr(counters),
                              torch.cuda.current_stream().cuda_stream)
    return rc, {"face": face, "absorbed": absorbed, "emitted": emitted,
                "counters": {n: int(v) for n, v in zip(N.COUNTER_NAMES, counters)}}


def _same(got, want, film, want_film):
    for key in ("face", "absorbed", "emitted"):
        assert np.array_equal(got[key], want[key]), key
    assert got["counters"] == want["counters"]
    assert torch.allclose(film, want_film, rtol=1e-5, atol=1e-6 * float(want_film.max()))


@pytest.mark.parametrize("form", ["wavefront", "wavefront_warp", "plain"])
def test_noalloc_render_matches_allocating_render_on_two_calls(form):
    require_gpu()
    sc = sg.cfg2_cornell_box(width=32, height=32, grid=32, n_paths=20000)
    n = sc["params"]["n_paths"]
    S = Scene(sc)
    want_film = S.render(form=form).clone()
    want = S.read()
    conc_t = torch.from_numpy(sc["medium"]["conc"]).cuda()
    solv_t = torch.from_numpy(sc["medium"]["solvent"]).cuda()
    film = torch.full_like(want_film, 123.0)
    for call in range(2):
        rc, got = _noalloc(sc, conc_t, solv_t, n, form, film)
        assert rc == N.FLR_OK, call
        _same(got, want, film, want_film)
    S.close()


def test_noalloc_homogeneous_medium_without_grids():
    require_gpu()
    sc = sg.cfg1_homogeneous_cube(n_paths=20000, film=32)
    S = Scene(sc)
    for form in ("wavefront_warp", "plain"):
        want_film = S.render(form=form).clone()
        want = S.read()
        film = torch.full_like(want_film, -1.0)
        for call in range(2):
            rc, got = _noalloc(sc, None, None, sc["params"]["n_paths"], form, film)
            assert rc == N.FLR_OK, (form, call)
            _same(got, want, film, want_film)
    S.close()


def test_noalloc_medium_without_mask_where_reads_are_skipped():
    """A light-sheet medium (grids, no solvent mask, sigma_s most of every majorant): both entry
    points launch the instances that take decisions without a grid read where a bound settles
    them, and must agree bit for bit."""
    require_gpu()
    sc = sg.cfg5_light_sheet(grid=32, width=32, height=32, n_blobs=40, n_paths=20000,
                             sigma_t_ref=20.0)
    S = Scene(sc)
    conc_t = torch.from_numpy(sc["medium"]["conc"]).cuda()
    for form in ("wavefront_warp", "plain"):
        want_film = S.render(form=form).clone()
        want = S.read()
        film = torch.full_like(want_film, 7.0)
        rc, got = _noalloc(sc, conc_t, None, sc["params"]["n_paths"], form, film)
        assert rc == N.FLR_OK, form
        _same(got, want, film, want_film)
    S.close()


def test_noalloc_rejects_grids_beyond_its_static_scratch():
    require_gpu()
    sc = sg.cfg4_adjoint(grid=65, width=8, height=8, n_paths=10)
    conc_t = torch.from_numpy(sc["medium"]["conc"]).cuda()
    film = torch.zeros((8, 8, sg.N_BINS), device="cuda")
    assert 65 ** 3 > N.FLR_NOALLOC_MAX_VOXELS
    rc, _ = _noalloc(sc, conc_t, None, 10, "plain", film)
    assert rc == N.FLR_ERR_ARG


@pytest.mark.parametrize("over", [{"paper_mode": 1}, {"skip_cell": 1}, {"macro_cell": 4},
                                  {"majorant_margin": 0.1}, {"hero": 2}])
def test_noalloc_rejects_settings_it_cannot_honour(over):
    require_gpu()
    sc = sg.cfg2_cornell_box(width=8, height=8, grid=16, n_paths=100)
    conc_t = torch.from_numpy(sc["medium"]["conc"]).cuda()
    solv_t = torch.from_numpy(sc["medium"]["solvent"]).cuda()
    film = torch.zeros((8, 8, sg.N_BINS), device="cuda")
    rc, _ = _noalloc(sc, conc_t, solv_t, 100, "wavefront_warp", film, **over)
    assert rc == N.FLR_ERR_ARG
    rc, _ = _noalloc(sc, conc_t, solv_t, 100, "wavefront_warp", film)
    assert rc == N.FLR_OK


def test_noalloc_reports_paths_cut_at_their_step_budget():
    require_gpu()
    sc = sg.cfg2_cornell_box(width=8, height=8, grid=16, n_paths=2000)
    conc_t = torch.from_numpy(sc["medium"]["conc"]).cuda()
    solv_t = torch.from_numpy(sc["medium"]["solvent"]).cuda()
    film = torch.zeros((8, 8, sg.N_BINS), device="cuda")
    rc, got = _noalloc(sc, conc_t, solv_t, 2000, "wavefront_warp", film, max_steps=1)
    assert rc == N.FLR_ERR_BUDGET
    assert got["counters"]["step_budget"] > 0
    # the next call starts from a clear error word
    rc, got = _noalloc(sc, conc_t, solv_t, 2000, "wavefront_warp", film)
    assert rc == N.FLR_OK and got["counters"]["step_budget"] == 0
