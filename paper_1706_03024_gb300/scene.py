"""Scene marshalling: a scene description dict (the layout scenegen documents) -> C-ABI calls.

PyTorch provides device memory and streams only. Grids are copied to CUDA tensors here; the
library's own kernels do every step of the transport.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import native as N

_KINDS = {"collimated": N.FLR_SOURCE_COLLIMATED, "lambertian": N.FLR_SOURCE_LAMBERTIAN}
_SENSORS = {"none": N.FLR_SENSOR_NONE, "ortho": N.FLR_SENSOR_ORTHO, "pinhole": N.FLR_SENSOR_PINHOLE}
_FORMS = {"plain": N.FLR_FORM_PLAIN, "wavefront": N.FLR_FORM_WAVEFRONT,
          "wavefront_warp": N.FLR_FORM_WAVEFRONT_WARP, "wavefront_pool": N.FLR_FORM_WAVEFRONT_POOL}


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def make_source(src):
    s = N.flr_source()
    s.kind = _KINDS[src["kind"]]
    s.origin[:] = src["origin"]
    s.eu[:] = src["eu"]
    s.ev[:] = src["ev"]
    s.dir[:] = src["dir"]
    lines = list(src["lines_nm"])
    if not 1 <= len(lines) <= N.FLR_MAX_LINES:
        raise ValueError("1..8 lines per source")
    s.n_lines = len(lines)
    for i, (lam, pw) in enumerate(zip(lines, src["power"])):
        s.lambda_nm[i] = float(lam)
        s.power[i] = float(pw)
    return s


def make_sensor(sn):
    c = N.flr_sensor()
    c.kind = _SENSORS[sn["kind"]]
    c.width = int(sn["width"])
    c.height = int(sn["height"])
    c.origin[:] = sn["origin"]
    c.U[:] = sn["U"]
    c.V[:] = sn["V"]
    c.view[:] = sn["view"]
    c.fov_y_deg = float(sn["fov_y_deg"])
    return c


class Scene:
    """One context holding one single-scene medium. Use render() / read()."""

    def __init__(self, scene, device=0, grids=None):
        """scene: scenegen dict. grids: optional dict of already-resident CUDA tensors
        {'conc': [D,nz,ny,nx] f32, 'solvent': [nz,ny,nx] u8} used instead of copying."""
        self.device = device
        self.desc = scene
        self.ctx = N.flr_create(device)
        self._keep = []
        sp, dy, md = scene["spectrum"], scene["dyes"], scene["medium"]
        self.B = int(sp["n_bins"])
        N.check(N.flr_set_spectrum(self.ctx, sp["lambda0"], sp["dlambda"], self.B), self.ctx,
                "flr_set_spectrum")
        self.set_dyes(dy)
        srcs = scene["sources"]
        arr = (N.flr_source * len(srcs))(*[make_source(s) for s in srcs])
        N.check(N.flr_set_sources(self.ctx, len(srcs), arr), self.ctx, "flr_set_sources")
        self.D = int(np.asarray(dy["eps"]).shape[0])
        self.set_medium(md, grids)
        self.sensor = scene["sensor"]
        N.check(N.flr_set_sensor(self.ctx, make_sensor(self.sensor)), self.ctx, "flr_set_sensor")
        self.film = None

    def set_dyes(self, dy):
        a = np.ascontiguousarray(dy["abs_shape"], np.float32)
        e = np.ascontiguousarray(dy["emit_spec"], np.float32)
        eps = np.ascontiguousarray(dy["eps"], np.float32)
        qy = np.ascontiguousarray(dy["qy"], np.float32)
        N.check(N.flr_set_dyes(self.ctx, eps.shape[0], _np_ptr(a), _np_ptr(e), _np_ptr(eps),
                               _np_ptr(qy)), self.ctx, "flr_set_dyes")

    def set_medium(self, md, grids=None, stream=None):
        """Upload a medium description; grids (CUDA tensors) may replace md's host arrays. With a
        stream, the upload is ordered on it (flr_set_medium_async) instead of the whole device."""
        m = N.flr_medium()
        m.lo[:] = md["lo"]
        m.hi[:] = md["hi"]
        D = self.D
        m.n_dyes = D
        for d in range(D):
            m.dye_ids[d] = d
        cu = np.asarray(md["conc_uniform"], np.float32)
        for d in range(D):
            m.conc_uniform[d] = float(cu[d]) if d < cu.shape[0] else 0.0
        dev = torch.device("cuda", self.device)
        conc_t = None
        solv_t = None
        if grids is not None:
            conc_t = grids.get("conc")
            solv_t = grids.get("solvent")
        else:
            if md.get("conc") is not None:
                conc_t = torch.from_numpy(np.ascontiguousarray(md["conc"], np.float32)).to(dev)
            if md.get("solvent") is not None:
                solv_t = torch.from_numpy(np.ascontiguousarray(md["solvent"], np.uint8)).to(dev)
        self.conc_t, self.solv_t = conc_t, solv_t
        if conc_t is not None:
            Dg, nz, ny, nx = conc_t.shape
            m.dims[:] = (nx, ny, nz)
            for d in range(D):
                m.conc[d] = conc_t[d].data_ptr()
        elif solv_t is not None:
            nz, ny, nx = solv_t.shape
            m.dims[:] = (nx, ny, nz)
        if solv_t is not None:
            m.solvent = solv_t.data_ptr()
        m.sigma_s = float(md["sigma_s"])
        m.sigma_a0 = float(md["sigma_a0"])
        m.wall_mask = int(md["wall_mask"])
        m.wall_albedo = float(md["wall_albedo"])
        m.ior = float(md.get("ior", 1.0))
        m.wall_gloss = float(md.get("wall_gloss", 0.0))
        m.wall_exponent = float(md.get("wall_exponent", 0.0))
        if stream is not None:
            N.check(N.flr_set_medium_async(self.ctx, m, stream.cuda_stream), self.ctx,
                    "flr_set_medium_async")
        else:
            N.check(N.flr_set_medium(self.ctx, m), self.ctx, "flr_set_medium")

    def film_tensor(self):
        sn = self.sensor
        if sn["kind"] == "none":
            return None
        if self.film is None:
            self.film = torch.zeros((sn["height"], sn["width"], self.B), dtype=torch.float32,
                                    device=torch.device("cuda", self.device))
        return self.film

    def set_medium_values(self, conc, sigma_s):
        """Re-upload the medium from a CUDA concentration tensor [D,nz,ny,nx] and a sigma_s."""
        md = dict(self.desc["medium"])
        md["sigma_s"] = float(sigma_s)
        self.desc = dict(self.desc)
        self.desc["medium"] = md
        self.set_medium(md, grids={"conc": conc, "solvent": self.solv_t})

    def _params(self, n_paths=None, path_offset=0, seed=None, medium_id=0, form="plain",
                analog=None, max_inelastic=None, n_rr=None, max_events=None, max_steps=None,
                accumulate=False, block_size=0, blocks_per_sm=0, regroup=0, macro_cell=0,
                majorant_margin=0.0, skip_cell=0, paper_mode=False, hero=0):
        pp = dict(self.desc["params"])
        for k, v in (("n_paths", n_paths), ("seed", seed), ("analog", analog),
                     ("max_inelastic", max_inelastic), ("n_rr", n_rr), ("max_events", max_events),
                     ("max_steps", max_steps)):
            if v is not None:
                pp[k] = v
        p = N.flr_params()
        p.n_paths = int(pp["n_paths"])
        p.path_offset = int(path_offset)
        p.seed = int(pp["seed"])
        p.medium_id = int(medium_id)
        p.n_rr = int(pp["n_rr"])
        p.max_inelastic = int(pp["max_inelastic"])
        p.analog = int(pp["analog"])
        p.form = _FORMS[form] if isinstance(form, str) else int(form)
        p.max_events = int(pp["max_events"])
        p.max_steps = int(pp.get("max_steps", 100_000_000))
        p.accumulate = 1 if accumulate else 0
        p.block_size = int(block_size)
        p.blocks_per_sm = int(blocks_per_sm)
        p.regroup_interval = int(regroup)
        p.macro_cell = int(macro_cell)
        p.skip_cell = int(skip_cell)
        p.majorant_margin = float(majorant_margin)
        p.paper_mode = 1 if paper_mode else 0
        p.hero = int(hero)
        return p

    def render(self, n_paths=None, path_offset=0, seed=None, medium_id=0, form="plain",
               analog=None, max_inelastic=None, n_rr=None, max_events=None, max_steps=None,
               film=True, path_events=None, accumulate=False, block_size=0, blocks_per_sm=0,
               regroup=0, macro_cell=0, majorant_margin=0.0, skip_cell=0, paper_mode=False,
               hero=0, stream=None):
        p = self._params(n_paths, path_offset, seed, medium_id, form, analog, max_inelastic, n_rr,
                         max_events, max_steps, accumulate, block_size, blocks_per_sm, regroup,
                         macro_cell, majorant_margin, skip_cell, paper_mode, hero)
        f = self.film_tensor() if film else None
        p.film = f.data_ptr() if f is not None else None
        p.path_events = path_events.data_ptr() if path_events is not None else None
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        N.check(N.flr_render(self.ctx, p, st.cuda_stream), self.ctx, "flr_render")
        return f

    def render_camera(self, n_paths=None, path_offset=0, seed=None, medium_id=0, analog=None,
                      n_rr=None, max_events=None, max_steps=None, accumulate=False, block_size=0,
                      form="wavefront_warp", stream=None):
        """The paper's camera-side estimator of its single-inelastic model (flr_render_camera):
        returns the film tensor [H, W, B] of fluorescence radiance; n_paths and path_offset must
        be multiples of W*H."""
        p = self._params(n_paths, path_offset, seed, medium_id, form, analog, None, n_rr,
                         max_events, max_steps, accumulate, block_size)
        f = self.film_tensor()
        p.film = f.data_ptr()
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        N.check(N.flr_render_camera(self.ctx, p, st.cuda_stream), self.ctx, "flr_render_camera")
        return f

    def adjoint(self, adj, grad_conc=None, grad_sigma_s=None, n_paths=None, path_offset=0,
                seed=None, medium_id=0, analog=None, max_inelastic=None, n_rr=None,
                max_events=None, max_steps=None, accumulate=False, block_size=0, macro_cell=0,
                majorant_margin=0.0, skip_cell=0, form="wavefront_warp", regroup=0, stream=None):
        """Path-replay gradient of sum(adj * film) for the paths render() traces with the same
        arguments; writes into grad_conc [D,nz,ny,nx] and grad_sigma_s [1] (CUDA f32 tensors).
        form "plain": one thread replays a whole path twice; "wavefront_warp" (or "wavefront"):
        two warp-regrouped passes, contributions first, then the gradients."""
        p = self._params(n_paths, path_offset, seed, medium_id, form, analog, max_inelastic,
                         n_rr, max_events, max_steps, accumulate, block_size, regroup=regroup,
                         macro_cell=macro_cell, majorant_margin=majorant_margin,
                         skip_cell=skip_cell)
        adj = adj.contiguous()
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        N.check(N.flr_adjoint(self.ctx, p, adj.data_ptr(),
                              grad_conc.data_ptr() if grad_conc is not None else None,
                              grad_sigma_s.data_ptr() if grad_sigma_s is not None else None,
                              st.cuda_stream), self.ctx, "flr_adjoint")

    def frozen_sums(self, adj, pert=(-1, 0, 0.0, 0.0), n_paths=None, path_offset=0, seed=None,
                    medium_id=0, majorant_margin=0.0, stream=None):
        """Per-path adjoint-weighted film contributions under the frozen-sampling estimator at the
        perturbed medium pert = (dye slot or -1, voxel, delta, d_sigma_s) (flr_debug_frozen_sums):
        an fp64 tensor [n_paths] for the paths adjoint() replays with the same arguments."""
        p = self._params(n_paths, path_offset, seed, medium_id, "plain",
                         majorant_margin=majorant_margin)
        out = torch.empty(int(p.n_paths), dtype=torch.float64,
                          device=torch.device("cuda", self.device))
        adj = adj.contiguous()
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        d, v, delta, ds = pert
        N.check(N.flr_debug_frozen_sums(self.ctx, p, adj.data_ptr(), -1 if d is None else d, v,
                                        delta, ds, out.data_ptr(), st.cuda_stream), self.ctx,
                "flr_debug_frozen_sums")
        return out

    def read(self, stream=None):
        B, D = self.B, self.D
        face = np.zeros((2, 6, B))
        absorbed = np.zeros((D + 1, B))
        emitted = np.zeros((max(D, 1), B))
        counters = np.zeros(N.FLR_NCOUNTERS, np.uint64)
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        N.check(N.flr_read_tallies(self.ctx, _np_ptr(face), _np_ptr(absorbed), _np_ptr(emitted),
                                   _np_ptr(counters), st.cuda_stream), self.ctx,
                "flr_read_tallies")
        return {"face": face, "absorbed": absorbed, "emitted": emitted[:D],
                "counters": {n: int(v) for n, v in zip(N.COUNTER_NAMES, counters)}}

    def status(self):
        return N.flr_status(self.ctx)

    def close(self):
        if self.ctx:
            N.flr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FluoroRender(torch.autograd.Function):
    """film = render(conc, sigma_s) through flr_render; backward is flr_adjoint (path replay of
    the same paths, gradient of the frozen-sampling estimator).

    Usage: film = FluoroRender.apply(conc, sigma_s, scene, opts) with conc a CUDA f32 tensor
    [D,nz,ny,nx], sigma_s a 0-d tensor, scene a Scene and opts the render keyword arguments
    (n_paths, seed, path_offset, form, ...; "adjoint_form" picks the replay's form)."""

    @staticmethod
    def forward(ctx, conc, sigma_s, scene, opts):
        # a majorant margin keeps the replay's null-collision scores bounded (default 10 %)
        opts = dict(opts)
        opts.setdefault("majorant_margin", 0.1)
        conc_c = conc.detach().contiguous()
        scene.set_medium_values(conc_c, float(sigma_s))
        film = scene.render(form=opts.get("form", "wavefront_warp"),
                            **{k: v for k, v in opts.items()
                               if k not in ("form", "adjoint_form")}).clone()
        ctx.save_for_backward(conc_c, sigma_s.detach())
        ctx.scene = scene
        ctx.opts = opts
        return film

    @staticmethod
    def backward(ctx, grad_film):
        conc, sigma_s = ctx.saved_tensors
        S = ctx.scene
        S.set_medium_values(conc, float(sigma_s))
        gc = torch.empty_like(conc) if ctx.needs_input_grad[0] else None
        gs = torch.empty(1, dtype=torch.float32, device=conc.device)
        opts = {k: v for k, v in ctx.opts.items() if k not in ("form", "regroup", "adjoint_form")}
        S.adjoint(grad_film.float(), gc, gs, form=ctx.opts.get("adjoint_form", "wavefront_warp"),
                  **opts)
        return gc, gs.reshape(()).to(sigma_s.dtype), None, None


class Batch:
    """Many independent media (scene dicts sharing one spectrum) in one persistent launch."""

    def __init__(self, scenes, device=0, seed=0, medium_id=0, n_rr=5, max_events=1_000_000,
                 max_inelastic=-1, analog=0, max_steps=10_000_000, block_size=0,
                 blocks_per_sm=0, path_offset=0):
        self.device = device
        self.ctx = N.flr_create(device)
        sp = scenes[0]["spectrum"]
        self.B = int(sp["n_bins"])
        self.M = len(scenes)
        N.check(N.flr_set_spectrum(self.ctx, sp["lambda0"], sp["dlambda"], self.B), self.ctx,
                "flr_set_spectrum")
        dev = torch.device("cuda", device)
        abs_rows, em_rows, eps, qy, srcs = [], [], [], [], []
        meds = (N.flr_medium * self.M)()
        self.grids = []
        n_paths = np.zeros(self.M, dtype=np.uint64)
        for i, sc in enumerate(scenes):
            dy, md = sc["dyes"], sc["medium"]
            D = int(np.asarray(dy["eps"]).shape[0])
            m = meds[i]
            m.n_dyes = D
            for d in range(D):
                m.dye_ids[d] = len(eps)
                abs_rows.append(np.asarray(dy["abs_shape"][d], np.float32))
                em_rows.append(np.asarray(dy["emit_spec"][d], np.float32))
                eps.append(float(dy["eps"][d]))
                qy.append(float(dy["qy"][d]))
            m.lo[:] = md["lo"]
            m.hi[:] = md["hi"]
            cu = np.asarray(md["conc_uniform"], np.float32)
            for d in range(D):
                m.conc_uniform[d] = float(cu[d]) if d < cu.shape[0] else 0.0
            if md.get("conc") is not None:
                g = torch.from_numpy(np.ascontiguousarray(md["conc"], np.float32)).to(dev)
                self.grids.append(g)
                _, nz, ny, nx = g.shape
                m.dims[:] = (nx, ny, nz)
                for d in range(D):
                    m.conc[d] = g[d].data_ptr()
            if md.get("solvent") is not None:
                sv = torch.from_numpy(np.ascontiguousarray(md["solvent"], np.uint8)).to(dev)
                self.grids.append(sv)
                nz, ny, nx = sv.shape
                m.dims[:] = (nx, ny, nz)
                m.solvent = sv.data_ptr()
            m.sigma_s = float(md["sigma_s"])
            m.sigma_a0 = float(md["sigma_a0"])
            m.wall_mask = int(md["wall_mask"])
            m.wall_albedo = float(md["wall_albedo"])
            m.ior = float(md.get("ior", 1.0))
            m.wall_gloss = float(md.get("wall_gloss", 0.0))
            m.wall_exponent = float(md.get("wall_exponent", 0.0))
            m.source_first = len(srcs)
            m.source_count = len(sc["sources"])
            srcs.extend(make_source(s) for s in sc["sources"])
            n_paths[i] = int(sc["params"]["n_paths"])
        a = np.ascontiguousarray(np.stack(abs_rows), np.float32)
        e = np.ascontiguousarray(np.stack(em_rows), np.float32)
        ep = np.ascontiguousarray(eps, np.float32)
        q = np.ascontiguousarray(qy, np.float32)
        N.check(N.flr_set_dyes(self.ctx, len(eps), _np_ptr(a), _np_ptr(e), _np_ptr(ep), _np_ptr(q)),
                self.ctx, "flr_set_dyes")
        arr = (N.flr_source * len(srcs))(*srcs)
        N.check(N.flr_set_sources(self.ctx, len(srcs), arr), self.ctx, "flr_set_sources")
        p = N.flr_params()
        p.n_paths = int(n_paths.sum())
        p.path_offset = int(path_offset)
        p.seed = int(seed)
        p.medium_id = int(medium_id)
        p.n_rr = int(n_rr)
        p.max_inelastic = int(max_inelastic)
        p.analog = int(analog)
        p.max_events = int(max_events)
        p.max_steps = int(max_steps)
        p.block_size = int(block_size)
        p.blocks_per_sm = int(blocks_per_sm)
        self.n_paths = n_paths
        self.media = meds
        N.check(N.flr_batch_prepare(self.ctx, self.M, meds, _np_ptr(n_paths), p), self.ctx,
                "flr_batch_prepare")

    def launch(self, stream=None):
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        N.check(N.flr_batch_launch(self.ctx, st.cuda_stream), self.ctx, "flr_batch_launch")

    def read(self, stream=None):
        B, M, MD = self.B, self.M, N.FLR_MAX_DYES_PER_MEDIUM
        face = np.zeros((M, 2, 6, B))
        absorbed = np.zeros((M, MD + 1, B))
        emitted = np.zeros((M, MD, B))
        counters = np.zeros(N.FLR_NCOUNTERS, np.uint64)
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        N.check(N.flr_batch_read(self.ctx, _np_ptr(face), _np_ptr(absorbed), _np_ptr(emitted),
                                 _np_ptr(counters), st.cuda_stream), self.ctx, "flr_batch_read")
        return {"face": face, "absorbed": absorbed, "emitted": emitted,
                "counters": {n: int(v) for n, v in zip(N.COUNTER_NAMES, counters)}}

    def close(self):
        if self.ctx:
            N.flr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
