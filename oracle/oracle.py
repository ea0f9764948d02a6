"""ctypes marshalling for the C oracle in fluoro_oracle.c (test infrastructure only).

build() compiles the oracle with gcc (-O2, OpenMP) into oracle/_build/; render() takes a scene
dict from scenegen and returns fp64 tallies normalised per launched path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fluoro_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

COUNTER_NAMES = [
    "paths", "events", "nulls", "escapes", "absorbed_dead", "rr_kills", "cap_hits", "step_budget",
    "connections", "vf_rejected", "wall_bounces", "emissions", "scatters", "dye_absorptions",
    "steps", "majorant_violations", "iface_reflections",
]

MAX_DYES = 4
MAX_EMITTERS = 32


class Emitter(C.Structure):
    _fields_ = [("kind", C.c_int), ("origin", C.c_double * 3), ("eu", C.c_double * 3),
                ("ev", C.c_double * 3), ("dir", C.c_double * 3), ("lambda_nm", C.c_double),
                ("power", C.c_double), ("group", C.c_int)]


class Sensor(C.Structure):
    _fields_ = [("kind", C.c_int), ("width", C.c_int), ("height", C.c_int),
                ("origin", C.c_double * 3), ("U", C.c_double * 3), ("V", C.c_double * 3),
                ("view", C.c_double * 3), ("fov_y_deg", C.c_double)]


class Scene(C.Structure):
    _fields_ = [
        ("n_bins", C.c_int), ("lambda0", C.c_double), ("dlambda", C.c_double),
        ("n_dyes", C.c_int), ("abs_shape", C.POINTER(C.c_float)),
        ("emit_spec", C.POINTER(C.c_float)), ("eps", C.POINTER(C.c_float)),
        ("qy", C.POINTER(C.c_float)),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("dims", C.c_int * 3),
        ("conc", C.POINTER(C.c_float)), ("conc_uniform", C.POINTER(C.c_float)),
        ("solvent", C.POINTER(C.c_uint8)), ("sigma_s", C.c_double), ("sigma_a0", C.c_double),
        ("wall_mask", C.c_int), ("wall_albedo", C.c_double),
        ("n_emitters", C.c_int), ("emitters", C.POINTER(Emitter)),
        ("sensor", Sensor),
        ("ior", C.c_double), ("wall_gloss", C.c_double), ("wall_exponent", C.c_double),
    ]


class Params(C.Structure):
    _fields_ = [("n_paths", C.c_uint64), ("path_offset", C.c_uint64), ("seed", C.c_uint32),
                ("medium_id", C.c_uint32), ("n_rr", C.c_int), ("max_inelastic", C.c_int),
                ("analog", C.c_int), ("n_threads", C.c_int), ("max_events", C.c_int64),
                ("max_steps", C.c_int64), ("majorant_scale", C.c_double), ("frozen", C.c_int),
                ("pert_dye", C.c_int), ("pert_voxel", C.c_int64), ("pert_delta", C.c_double),
                ("pert_sigma_s", C.c_double), ("macro_cell", C.c_int), ("skip_cell", C.c_int),
                ("paper_mode", C.c_int), ("hero", C.c_int)]


class Result(C.Structure):
    _fields_ = [("face", C.POINTER(C.c_double)), ("absorbed", C.POINTER(C.c_double)),
                ("emitted", C.POINTER(C.c_double)), ("film", C.POINTER(C.c_double)),
                ("counters", C.POINTER(C.c_uint64)), ("path_events", C.POINTER(C.c_uint32))]


def build(force=False):
    """Compile the oracle with gcc into oracle/_build/liboracle.so (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC,
           "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            L.or_render.argtypes = [C.POINTER(Scene), C.POINTER(Params), C.POINTER(Result)]
            L.or_render.restype = C.c_int
            L.or_philox.argtypes = [C.c_uint32, C.c_uint32, C.c_void_p, C.c_int64, C.c_void_p]
            L.or_philox.restype = None
            L.or_sample_emission.argtypes = [C.POINTER(Scene), C.c_int, C.c_void_p, C.c_int64,
                                             C.c_void_p]
            L.or_sample_emission.restype = C.c_int
            L.or_iso_dir.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
            L.or_iso_dir.restype = None
            L.or_cosine_dir.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_double,
                                        C.c_void_p]
            L.or_cosine_dir.restype = None
            L.or_optical_depth.argtypes = [C.POINTER(Scene), C.c_void_p, C.c_void_p, C.c_double,
                                           C.c_int]
            L.or_optical_depth.restype = C.c_double
            L.or_majorant.argtypes = [C.POINTER(Scene), C.c_void_p]
            L.or_majorant.restype = None
            L.or_sigma_t_at.argtypes = [C.POINTER(Scene), C.c_void_p, C.c_int64, C.c_int,
                                        C.c_void_p, C.c_void_p]
            L.or_sigma_t_at.restype = None
            L.or_adjoint.argtypes = [C.POINTER(Scene), C.POINTER(Params), C.c_void_p,
                                     C.c_void_p, C.c_void_p]
            L.or_adjoint.restype = C.c_int
            L.or_render_camera.argtypes = [C.POINTER(Scene), C.POINTER(Params), C.c_void_p,
                                           C.c_void_p]
            L.or_render_camera.restype = C.c_int
            _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class _SceneHolder:
    """Keeps the numpy buffers alive while the C scene points into them."""

    def __init__(self, scene):
        sp, dy, md = scene["spectrum"], scene["dyes"], scene["medium"]
        self.abs_shape = _f32(dy["abs_shape"])
        self.emit_spec = _f32(dy["emit_spec"])
        self.eps = _f32(dy["eps"])
        self.qy = _f32(dy["qy"])
        D = int(self.eps.shape[0])
        if D > MAX_DYES:
            raise ValueError("oracle supports at most 4 dyes per medium")
        self.conc = _f32(md["conc"]) if md.get("conc") is not None else None
        self.conc_uniform = _f32(md["conc_uniform"]) if md.get("conc_uniform") is not None \
            else np.zeros(max(D, 1), np.float32)
        self.solvent = (np.ascontiguousarray(md["solvent"], dtype=np.uint8)
                        if md.get("solvent") is not None else None)
        ems = []
        for gi, src in enumerate(scene["sources"]):
            for lam, pw in zip(src["lines_nm"], src["power"]):
                e = Emitter()
                e.group = gi
                e.kind = 0 if src["kind"] == "collimated" else 1
                e.origin[:] = src["origin"]
                e.eu[:] = src["eu"]
                e.ev[:] = src["ev"]
                e.dir[:] = src["dir"]
                e.lambda_nm = float(lam)
                e.power = float(pw)
                ems.append(e)
        if not ems or len(ems) > MAX_EMITTERS:
            raise ValueError("need 1..32 emitter lines")
        self.emitters = (Emitter * len(ems))(*ems)
        s = Scene()
        s.n_bins = int(sp["n_bins"])
        s.lambda0 = float(sp["lambda0"])
        s.dlambda = float(sp["dlambda"])
        s.n_dyes = D
        s.abs_shape = _ptr(self.abs_shape, C.c_float)
        s.emit_spec = _ptr(self.emit_spec, C.c_float)
        s.eps = _ptr(self.eps, C.c_float)
        s.qy = _ptr(self.qy, C.c_float)
        s.lo[:] = md["lo"]
        s.hi[:] = md["hi"]
        if md.get("dims") is not None and self.conc is not None:
            s.dims[:] = md["dims"]
        elif self.solvent is not None:
            nz, ny, nx = self.solvent.shape
            s.dims[:] = (nx, ny, nz)
        else:
            s.dims[:] = (0, 0, 0)
        s.conc = _ptr(self.conc, C.c_float) if self.conc is not None else None
        s.conc_uniform = _ptr(self.conc_uniform, C.c_float)
        s.solvent = _ptr(self.solvent, C.c_uint8) if self.solvent is not None else None
        s.sigma_s = float(md["sigma_s"])
        s.sigma_a0 = float(md["sigma_a0"])
        s.wall_mask = int(md["wall_mask"])
        s.wall_albedo = float(md["wall_albedo"])
        s.ior = float(md.get("ior", 1.0))
        s.wall_gloss = float(md.get("wall_gloss", 0.0))
        s.wall_exponent = float(md.get("wall_exponent", 0.0))
        s.n_emitters = len(ems)
        s.emitters = C.cast(self.emitters, C.POINTER(Emitter))
        sn = scene["sensor"]
        kinds = {"none": 0, "ortho": 1, "pinhole": 2}
        s.sensor.kind = kinds[sn["kind"]]
        s.sensor.width = int(sn["width"])
        s.sensor.height = int(sn["height"])
        s.sensor.origin[:] = sn["origin"]
        s.sensor.U[:] = sn["U"]
        s.sensor.V[:] = sn["V"]
        s.sensor.view[:] = sn["view"]
        s.sensor.fov_y_deg = float(sn["fov_y_deg"])
        self.scene = s
        self.n_dyes = D
        self.n_bins = s.n_bins


def render(scene, n_paths=None, path_offset=0, seed=None, medium_id=0, n_threads=0,
           analog=None, max_inelastic=None, n_rr=None, max_events=None, max_steps=None,
           film=True, path_events=False, majorant_scale=1.0, frozen=False, pert=None,
           macro_cell=0, skip_cell=0, paper_mode=False, hero=0):
    """Run the oracle; returns a dict of fp64 tallies normalised per launched path:
    face [2,6,B], absorbed [D+1,B], emitted [D,B], film [H,W,B] (or None), counters (dict),
    path_events u32[n] (or None).
    pert = (dye, voxel, delta, d_sigma_s) evaluates the scene with that perturbation (dye None for
    none); with frozen=True the decisions are still sampled in the unperturbed scene and every
    tally carries the likelihood ratio of the decisions before it.
    paper_mode=True: the paper's single-inelastic model (uncollided excitation, one emission,
    fluorescence-only film).
    hero=C (1..4): hero-wavelength paths carrying up to C wavelengths (spectral MIS)."""
    L = lib()
    h = _SceneHolder(scene)
    p = _params(scene, n_paths, path_offset, seed, medium_id, n_threads, analog, max_inelastic,
                n_rr, max_events, max_steps, majorant_scale, frozen, pert)
    p.macro_cell = int(macro_cell)
    p.skip_cell = int(skip_cell)
    p.paper_mode = 1 if paper_mode else 0
    p.hero = int(hero)
    return _render(L, h, scene, p, film, path_events)


def render_camera(scene, n_paths, path_offset=0, seed=None, medium_id=0, n_threads=0,
                  analog=None, n_rr=None, max_events=None, max_steps=None):
    """Camera-side estimator of the paper's single-inelastic model: returns
    {"film": [H,W,B] fluorescence radiance per unit source power, "counters": dict}. n_paths and
    path_offset must be multiples of W*H."""
    L = lib()
    h = _SceneHolder(scene)
    p = _params(scene, n_paths, path_offset, seed, medium_id, n_threads, analog, None, n_rr,
                max_events, max_steps, 1.0, False, None)
    sn = scene["sensor"]
    film = np.zeros((sn["height"], sn["width"], h.n_bins))
    counters = np.zeros(len(COUNTER_NAMES), dtype=np.uint64)
    rc = L.or_render_camera(C.byref(h.scene), C.byref(p), film.ctypes.data, counters.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle camera render rejected the scene (rc={rc})")
    return {"film": film, "counters": {n: int(v) for n, v in zip(COUNTER_NAMES, counters)}}


def _params(scene, n_paths, path_offset, seed, medium_id, n_threads, analog, max_inelastic, n_rr,
            max_events, max_steps, majorant_scale, frozen, pert):
    pp = dict(scene["params"])
    for k, v in (("n_paths", n_paths), ("seed", seed), ("analog", analog),
                 ("max_inelastic", max_inelastic), ("n_rr", n_rr), ("max_events", max_events),
                 ("max_steps", max_steps)):
        if v is not None:
            pp[k] = v
    p = Params()
    p.n_paths = int(pp["n_paths"])
    p.path_offset = int(path_offset)
    p.seed = int(pp["seed"])
    p.medium_id = int(medium_id)
    p.n_rr = int(pp["n_rr"])
    p.max_inelastic = int(pp["max_inelastic"])
    p.analog = int(pp["analog"])
    p.n_threads = int(n_threads)
    p.max_events = int(pp["max_events"])
    p.max_steps = int(pp.get("max_steps", 100_000_000))
    p.majorant_scale = float(majorant_scale)
    p.frozen = 1 if frozen else 0
    p.pert_dye = -1 if pert is None or pert[0] is None else int(pert[0])
    p.pert_voxel = 0 if pert is None or pert[0] is None else int(pert[1])
    p.pert_delta = 0.0 if pert is None or pert[0] is None else float(pert[2])
    p.pert_sigma_s = 0.0 if pert is None else float(pert[3] if len(pert) > 3 else 0.0)
    return p


def _render(L, h, scene, p, film, path_events):
    B, D = h.n_bins, h.n_dyes
    face = np.zeros((2, 6, B))
    absorbed = np.zeros((D + 1, B))
    emitted = np.zeros((max(D, 1), B))
    counters = np.zeros(len(COUNTER_NAMES), dtype=np.uint64)
    sn = scene["sensor"]
    fl = None
    if film and sn["kind"] != "none":
        fl = np.zeros((sn["height"], sn["width"], B))
    pe = np.zeros(p.n_paths, dtype=np.uint32) if path_events else None
    r = Result()
    r.face = _ptr(face, C.c_double)
    r.absorbed = _ptr(absorbed, C.c_double)
    r.emitted = _ptr(emitted, C.c_double)
    r.film = _ptr(fl, C.c_double) if fl is not None else None
    r.counters = _ptr(counters, C.c_uint64)
    r.path_events = _ptr(pe, C.c_uint32) if pe is not None else None
    rc = L.or_render(C.byref(h.scene), C.byref(p), C.byref(r))
    if rc != 0:
        raise ValueError(f"oracle rejected the scene (rc={rc})")
    return {"face": face, "absorbed": absorbed, "emitted": emitted[:D], "film": fl,
            "counters": {n: int(v) for n, v in zip(COUNTER_NAMES, counters)},
            "path_events": pe}


def philox(seed, medium, ctr):
    """Philox4x32-10 blocks for counters ctr u32[n,4] under key (seed, medium) -> u32[n,4]."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(ctr)
    lib().or_philox(int(seed), int(medium), ctr.ctypes.data, ctr.shape[0], out.ctypes.data)
    return out


def sample_emission(scene, dye, u):
    h = _SceneHolder(scene)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(u.shape[0], dtype=np.int32)
    rc = lib().or_sample_emission(C.byref(h.scene), int(dye), u.ctypes.data, u.shape[0],
                                  out.ctypes.data)
    if rc != 0:
        raise ValueError("bad dye index")
    return out


def iso_dir(u1, u2):
    u1 = np.ascontiguousarray(u1, dtype=np.float64)
    u2 = np.ascontiguousarray(u2, dtype=np.float64)
    out = np.zeros((u1.shape[0], 3))
    lib().or_iso_dir(u1.ctypes.data, u2.ctypes.data, u1.shape[0], out.ctypes.data)
    return out


def cosine_dir(u1, u2, axis, sign):
    u1 = np.ascontiguousarray(u1, dtype=np.float64)
    u2 = np.ascontiguousarray(u2, dtype=np.float64)
    out = np.zeros((u1.shape[0], 3))
    lib().or_cosine_dir(u1.ctypes.data, u2.ctypes.data, u1.shape[0], int(axis), float(sign),
                        out.ctypes.data)
    return out


def optical_depth(scene, x0, w, L, bin_index):
    h = _SceneHolder(scene)
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    return float(lib().or_optical_depth(C.byref(h.scene), x0.ctypes.data, w.ctypes.data,
                                        float(L), int(bin_index)))


def sigma_t_at(scene, pts, bin_index):
    """sigma_t at points [n, 3] in bin bin_index by the tracking's nearest-voxel lookup, and the
    row-major voxel index read (-1 for a medium without grids)."""
    h = _SceneHolder(scene)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    n = pts.shape[0]
    sig = np.zeros(n)
    vox = np.zeros(n, dtype=np.int64)
    lib().or_sigma_t_at(C.byref(h.scene), pts.ctypes.data, C.c_int64(n), int(bin_index),
                        sig.ctypes.data, vox.ctypes.data)
    return sig, vox


def majorant(scene):
    h = _SceneHolder(scene)
    out = np.zeros(h.n_bins)
    lib().or_majorant(C.byref(h.scene), out.ctypes.data)
    return out


def adjoint(scene, adj, n_paths=None, path_offset=0, seed=None, medium_id=0, n_threads=0,
            analog=None, max_inelastic=None, n_rr=None, max_events=None, max_steps=None,
            majorant_scale=1.0, macro_cell=0, skip_cell=0):
    """Reference gradient of sum(adj * film) over the same paths render() traces:
    returns (grad_conc [D,nz,ny,nx] or None, grad_sigma_s)."""
    L = lib()
    h = _SceneHolder(scene)
    p = _params(scene, n_paths, path_offset, seed, medium_id, n_threads, analog, max_inelastic,
                n_rr, max_events, max_steps, majorant_scale, False, None)
    p.macro_cell = int(macro_cell)
    p.skip_cell = int(skip_cell)
    adj = np.ascontiguousarray(adj, dtype=np.float64)
    sn = scene["sensor"]
    assert adj.shape == (sn["height"], sn["width"], h.n_bins)
    gc = None
    if h.conc is not None:
        gc = np.zeros(h.conc.shape, dtype=np.float64)
    gs = np.zeros(1, dtype=np.float64)
    rc = L.or_adjoint(C.byref(h.scene), C.byref(p), adj.ctypes.data,
                      gc.ctypes.data if gc is not None else None, gs.ctypes.data)
    if rc != 0:
        raise ValueError("oracle adjoint rejected the scene")
    return gc, float(gs[0])
