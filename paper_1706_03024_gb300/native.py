"""ctypes binding of the C ABI in include/fluoro.h (argument marshalling only).

Every function here has the C entry point's name and forwards to it; all compute runs in the
sm_103a kernels of libfluoro.so. The library is built in-tree by build.py; if it is missing this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

FLR_OK = 0
FLR_ERR_ARG = -1
FLR_ERR_CUDA = -2
FLR_ERR_OOM = -3
FLR_ERR_BUDGET = -4
FLR_ERR_STATE = -5

FLR_MAX_BINS = 128
FLR_MAX_DYES = 1024
FLR_MAX_DYES_PER_MEDIUM = 4
FLR_MAX_SOURCES = 65536
FLR_MAX_LINES = 8
FLR_MAX_EMITTERS = 32
FLR_NCOUNTERS = 21
FLR_NOALLOC_MAX_VOXELS = 1 << 18

FLR_SOURCE_COLLIMATED = 0
FLR_SOURCE_LAMBERTIAN = 1
FLR_SENSOR_NONE = 0
FLR_SENSOR_ORTHO = 1
FLR_SENSOR_PINHOLE = 2
FLR_FORM_PLAIN = 0
FLR_FORM_WAVEFRONT = 1
FLR_FORM_WAVEFRONT_WARP = 2
FLR_FORM_WAVEFRONT_POOL = 3

COUNTER_NAMES = [
    "paths", "events", "nulls", "escapes", "absorbed_dead", "rr_kills", "cap_hits", "step_budget",
    "connections", "vf_rejected", "wall_bounces", "emissions", "scatters", "dye_absorptions",
    "steps", "majorant_violations", "connect_steps", "connect_budget", "nonfinite", "cell_walks",
    "iface_reflections",
]

FLR_ERR_CHECK = -6
ERROR_NAMES = {FLR_OK: "FLR_OK", FLR_ERR_ARG: "FLR_ERR_ARG", FLR_ERR_CUDA: "FLR_ERR_CUDA",
               FLR_ERR_OOM: "FLR_ERR_OOM", FLR_ERR_BUDGET: "FLR_ERR_BUDGET",
               FLR_ERR_STATE: "FLR_ERR_STATE", FLR_ERR_CHECK: "FLR_ERR_CHECK"}


class flr_source(C.Structure):
    _fields_ = [("kind", C.c_int), ("origin", C.c_float * 3), ("eu", C.c_float * 3),
                ("ev", C.c_float * 3), ("dir", C.c_float * 3), ("n_lines", C.c_int),
                ("lambda_nm", C.c_float * FLR_MAX_LINES), ("power", C.c_float * FLR_MAX_LINES)]


class flr_medium(C.Structure):
    _fields_ = [("lo", C.c_float * 3), ("hi", C.c_float * 3), ("dims", C.c_int * 3),
                ("n_dyes", C.c_int), ("dye_ids", C.c_int * FLR_MAX_DYES_PER_MEDIUM),
                ("conc", C.c_void_p * FLR_MAX_DYES_PER_MEDIUM),
                ("conc_uniform", C.c_float * FLR_MAX_DYES_PER_MEDIUM),
                ("solvent", C.c_void_p), ("sigma_s", C.c_float), ("sigma_a0", C.c_float),
                ("wall_mask", C.c_int), ("wall_albedo", C.c_float),
                ("source_first", C.c_int), ("source_count", C.c_int), ("ior", C.c_float),
                ("wall_gloss", C.c_float), ("wall_exponent", C.c_float)]


class flr_sensor(C.Structure):
    _fields_ = [("kind", C.c_int), ("width", C.c_int), ("height", C.c_int),
                ("origin", C.c_float * 3), ("U", C.c_float * 3), ("V", C.c_float * 3),
                ("view", C.c_float * 3), ("fov_y_deg", C.c_float)]


class flr_params(C.Structure):
    _fields_ = [("n_paths", C.c_uint64), ("path_offset", C.c_uint64), ("seed", C.c_uint32),
                ("medium_id", C.c_uint32), ("n_rr", C.c_int), ("max_inelastic", C.c_int),
                ("analog", C.c_int), ("form", C.c_int), ("max_events", C.c_int64),
                ("max_steps", C.c_int64), ("film", C.c_void_p), ("path_events", C.c_void_p),
                ("accumulate", C.c_int), ("block_size", C.c_int), ("blocks_per_sm", C.c_int),
                ("regroup_interval", C.c_int), ("macro_cell", C.c_int),
                ("skip_cell", C.c_int), ("majorant_margin", C.c_float), ("paper_mode", C.c_int),
                ("hero", C.c_int)]


# name -> (restype, argtypes); every symbol include/fluoro.h declares
SIGNATURES = {
    "flr_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "flr_destroy": (None, [C.c_void_p]),
    "flr_set_spectrum": (C.c_int, [C.c_void_p, C.c_float, C.c_float, C.c_int]),
    "flr_set_dyes": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p]),
    "flr_set_sources": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(flr_source)]),
    "flr_set_medium": (C.c_int, [C.c_void_p, C.POINTER(flr_medium)]),
    "flr_set_medium_async": (C.c_int, [C.c_void_p, C.POINTER(flr_medium), C.c_void_p]),
    "flr_set_sensor": (C.c_int, [C.c_void_p, C.POINTER(flr_sensor)]),
    "flr_render": (C.c_int, [C.c_void_p, C.POINTER(flr_params), C.c_void_p]),
    "flr_render_camera": (C.c_int, [C.c_void_p, C.POINTER(flr_params), C.c_void_p]),
    "flr_read_tallies": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p]),
    "flr_adjoint": (C.c_int, [C.c_void_p, C.POINTER(flr_params), C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_void_p]),
    "flr_debug_frozen_sums": (C.c_int, [C.c_void_p, C.POINTER(flr_params), C.c_void_p, C.c_int,
                                        C.c_int64, C.c_float, C.c_float, C.c_void_p, C.c_void_p]),
    "flr_batch_prepare": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(flr_medium), C.c_void_p,
                                    C.POINTER(flr_params)]),
    "flr_batch_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "flr_batch_read": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p]),
    "flr_render_batch": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(flr_medium), C.c_void_p,
                                   C.POINTER(flr_params), C.c_void_p]),
    "flr_render_noalloc": (C.c_int, [C.c_float, C.c_float, C.c_int, C.c_int, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(flr_medium),
                                     C.c_int, C.POINTER(flr_source), C.POINTER(flr_sensor),
                                     C.POINTER(flr_params), C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p]),
    "flr_status": (C.c_int, [C.c_void_p]),
    "flr_last_error": (C.c_char_p, [C.c_void_p]),
    "flr_debug_philox": (C.c_int, [C.c_uint32, C.c_uint32, C.c_void_p, C.c_int64, C.c_void_p,
                                   C.c_void_p]),
    "flr_debug_sample_emission": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64,
                                            C.c_void_p, C.c_void_p]),
    "flr_debug_sigma_t": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "flr_debug_fail_alloc": (C.c_int, [C.c_int64]),
    "flr_checked_build": (C.c_int, []),
    "flr_debug_check": (C.c_int, [C.c_int64, C.c_int64, C.c_void_p]),
}

_lock = threading.Lock()
_lib = None


def library_path():
    """libfluoro.so, or libfluoro_checked.so when the environment sets FLR_CHECKED=1 (the build
    that tests every device index before its access)."""
    return _build.LIB_CHECKED if os.environ.get("FLR_CHECKED") == "1" else _build.LIB


def load(build_if_missing=False):
    """Load libfluoro.so (raises if it is not built; never substitutes another implementation)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                if build_if_missing:
                    _build.build(checked=path == _build.LIB_CHECKED)
                else:
                    raise RuntimeError(
                        f"{path} is missing: build it with `python -m paper_1706_03024_gb300.build`"
                        " (the CUDA extension is required; there is no CPU path)")
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class FluoroError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(rc, ctx=None, what=""):
    if rc != FLR_OK:
        msg = what
        if ctx:
            m = load().flr_last_error(ctx)
            msg = f"{what}: {m.decode() if m else ''}"
        raise FluoroError(rc, msg)
    return rc


# Same-name forwards -------------------------------------------------------------------------

def flr_create(device=0):
    ctx = C.c_void_p()
    check(load().flr_create(C.byref(ctx), int(device)), None, "flr_create")
    return ctx


def flr_destroy(ctx):
    load().flr_destroy(ctx)


def flr_set_spectrum(ctx, lambda0_nm, dlambda_nm, n_bins):
    return load().flr_set_spectrum(ctx, float(lambda0_nm), float(dlambda_nm), int(n_bins))


def flr_set_dyes(ctx, n, abs_shape_ptr, emit_spec_ptr, eps_ptr, qy_ptr):
    return load().flr_set_dyes(ctx, int(n), abs_shape_ptr, emit_spec_ptr, eps_ptr, qy_ptr)


def flr_set_sources(ctx, n, sources):
    return load().flr_set_sources(ctx, int(n), sources)


def flr_set_medium(ctx, medium):
    return load().flr_set_medium(ctx, C.byref(medium))


def flr_set_medium_async(ctx, medium, stream):
    return load().flr_set_medium_async(ctx, C.byref(medium), stream)


def flr_set_sensor(ctx, sensor):
    return load().flr_set_sensor(ctx, C.byref(sensor))


def flr_render(ctx, params, stream=0):
    return load().flr_render(ctx, C.byref(params), C.c_void_p(int(stream)))


def flr_render_camera(ctx, params, stream=0):
    return load().flr_render_camera(ctx, C.byref(params), C.c_void_p(int(stream)))


def flr_read_tallies(ctx, face_ptr, absorbed_ptr, emitted_ptr, counters_ptr, stream=0):
    return load().flr_read_tallies(ctx, face_ptr, absorbed_ptr, emitted_ptr, counters_ptr,
                                   C.c_void_p(int(stream)))


def flr_status(ctx):
    return load().flr_status(ctx)


def flr_last_error(ctx):
    m = load().flr_last_error(ctx)
    return m.decode() if m else ""


def flr_debug_philox(seed, medium, ctr_ptr, n, out_ptr, stream=0):
    return load().flr_debug_philox(int(seed), int(medium), ctr_ptr, int(n), out_ptr,
                                   C.c_void_p(int(stream)))


def flr_checked_build():
    return load().flr_checked_build()


def flr_debug_check(index, bound, stream=0):
    return load().flr_debug_check(int(index), int(bound), C.c_void_p(int(stream)))


def flr_debug_sample_emission(ctx, dye, u_ptr, n, out_ptr, stream=0):
    return load().flr_debug_sample_emission(ctx, int(dye), u_ptr, int(n), out_ptr,
                                            C.c_void_p(int(stream)))


def flr_debug_fail_alloc(k):
    return load().flr_debug_fail_alloc(int(k))


def flr_debug_sigma_t(ctx, points_ptr, n, bin_index, sigma_ptr, voxel_ptr=None, stream=0):
    return load().flr_debug_sigma_t(ctx, points_ptr, int(n), int(bin_index), sigma_ptr, voxel_ptr,
                                    C.c_void_p(int(stream)))


def flr_adjoint(ctx, params, adj_ptr, grad_conc_ptr, grad_sigma_s_ptr, stream=0):
    return load().flr_adjoint(ctx, C.byref(params), adj_ptr, grad_conc_ptr, grad_sigma_s_ptr,
                              C.c_void_p(int(stream)))


def flr_debug_frozen_sums(ctx, params, adj_ptr, pert_dye, pert_voxel, pert_delta, pert_sigma_s,
                          out_ptr, stream=0):
    return load().flr_debug_frozen_sums(ctx, C.byref(params), adj_ptr, int(pert_dye),
                                        int(pert_voxel), float(pert_delta), float(pert_sigma_s),
                                        out_ptr, C.c_void_p(int(stream)))


def flr_batch_prepare(ctx, n_media, media, n_paths_ptr, params):
    return load().flr_batch_prepare(ctx, int(n_media), media, n_paths_ptr, C.byref(params))


def flr_batch_launch(ctx, stream=0):
    return load().flr_batch_launch(ctx, C.c_void_p(int(stream)))


def flr_batch_read(ctx, face_ptr, absorbed_ptr, emitted_ptr, counters_ptr, stream=0):
    return load().flr_batch_read(ctx, face_ptr, absorbed_ptr, emitted_ptr, counters_ptr,
                                 C.c_void_p(int(stream)))


def flr_render_batch(ctx, n_media, media, n_paths_ptr, params, stream=0):
    return load().flr_render_batch(ctx, int(n_media), media, n_paths_ptr, C.byref(params),
                                   C.c_void_p(int(stream)))


def flr_render_noalloc(lambda0_nm, dlambda_nm, n_bins, n_dyes, abs_shape_ptr, emit_spec_ptr,
                       eps_ptr, qy_ptr, medium, n_sources, sources, sensor, params, face_ptr,
                       absorbed_ptr, emitted_ptr, counters_ptr, stream=0):
    """Single-scene render that allocates no device memory (see include/fluoro.h)."""
    return load().flr_render_noalloc(float(lambda0_nm), float(dlambda_nm), int(n_bins),
                                     int(n_dyes), abs_shape_ptr, emit_spec_ptr, eps_ptr, qy_ptr,
                                     C.byref(medium), int(n_sources), sources,
                                     C.byref(sensor) if sensor is not None else None,
                                     C.byref(params), face_ptr, absorbed_ptr, emitted_ptr,
                                     counters_ptr, C.c_void_p(int(stream)))
