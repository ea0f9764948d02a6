"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module builds scene *descriptions* only: spectra sampled at bin centres, voxel grids,
source and sensor geometry, path counts. It holds none of the method's arithmetic (no CDFs,
majorants, tracking, tallies); each side derives those itself.

The paper's measured dye spectra (Alexa Fluor, Sec. 5) are not available, so every dye is a
Gaussian absorption band and a Gaussian emission band, the shape the paper's Fig. 2 sketches for a
polyatomic fluorophore. Scenes mirror the paper's workloads: dyes dissolved in a strongly
scattering solvent (Sec. 5), spheres of dye (Fig. 1), monochromatic lines at each excitation peak.

Scene dict layout (all arrays numpy, C-contiguous):
    spectrum: lambda0 (nm), dlambda (nm), n_bins
    dyes:     abs_shape f32[D,B] (peak 1), emit_spec f32[D,B], eps f32[D] (napierian cm^-1 per unit
              concentration at the absorption peak), qy f32[D]
    medium:   lo, hi (cm), dims (nx,ny,nz) or None, conc f32[D,nz,ny,nx] or None,
              conc_uniform f32[D], solvent u8[nz,ny,nx] or None, sigma_s, sigma_a0 (cm^-1),
              wall_mask (bit f = face f is a Lambertian wall; faces -x,+x,-y,+y,-z,+z), wall_albedo;
              optional: ior (refractive index of the solution, > 1 makes the open faces smooth
              dielectric interfaces; default 1), wall_gloss (glossy share g of the walls' BRDF,
              default 0), wall_exponent (Phong exponent of the glossy lobe)
    sources:  list of dict(kind 'collimated'|'lambertian', origin, eu, ev, dir, lines_nm, power)
    sensor:   dict(kind 'none'|'ortho'|'pinhole', width, height, origin, U, V, view, fov_y_deg)
    params:   n_paths, seed, n_rr, max_events, max_inelastic, analog
"""
from __future__ import annotations

import math

import numpy as np

LAMBDA0 = 380.0
DLAMBDA = 5.0
N_BINS = 81

FACE_NX, FACE_PX, FACE_NY, FACE_PY, FACE_NZ, FACE_PZ = range(6)


def bin_centres(n_bins=N_BINS, lambda0=LAMBDA0, dlambda=DLAMBDA):
    return lambda0 + dlambda * np.arange(n_bins, dtype=np.float64)


def gaussian_band(peak_nm, sigma_nm, n_bins=N_BINS, lambda0=LAMBDA0, dlambda=DLAMBDA):
    """Gaussian evaluated at bin centres, peak value 1."""
    lam = bin_centres(n_bins, lambda0, dlambda)
    return np.exp(-0.5 * ((lam - peak_nm) / sigma_nm) ** 2).astype(np.float32)


def make_dyes(abs_peaks, abs_sigmas, em_peaks, em_sigmas, eps, qy, n_bins=N_BINS):
    D = len(abs_peaks)
    a = np.stack([gaussian_band(abs_peaks[d], abs_sigmas[d], n_bins) for d in range(D)])
    e = np.stack([gaussian_band(em_peaks[d], em_sigmas[d], n_bins) for d in range(D)])
    return {
        "abs_shape": np.ascontiguousarray(a, dtype=np.float32),
        "emit_spec": np.ascontiguousarray(e, dtype=np.float32),
        "eps": np.asarray(eps, dtype=np.float32).reshape(D),
        "qy": np.asarray(qy, dtype=np.float32).reshape(D),
    }


def spectrum():
    return {"lambda0": LAMBDA0, "dlambda": DLAMBDA, "n_bins": N_BINS}


def homogeneous_medium(n_dyes, conc=1.0, sigma_s=0.0, sigma_a0=0.0, lo=(0, 0, 0), hi=(1, 1, 1),
                       wall_mask=0, wall_albedo=0.0):
    return {
        "lo": tuple(float(v) for v in lo), "hi": tuple(float(v) for v in hi), "dims": None,
        "conc": None, "conc_uniform": np.full(n_dyes, conc, dtype=np.float32),
        "solvent": None, "sigma_s": float(sigma_s), "sigma_a0": float(sigma_a0),
        "wall_mask": int(wall_mask), "wall_albedo": float(wall_albedo),
    }


def grid_medium(conc, solvent=None, sigma_s=0.0, sigma_a0=0.0, lo=(0, 0, 0), hi=(1, 1, 1),
                wall_mask=0, wall_albedo=0.0):
    conc = np.ascontiguousarray(conc, dtype=np.float32)
    D, nz, ny, nx = conc.shape
    if solvent is not None:
        solvent = np.ascontiguousarray(solvent, dtype=np.uint8)
        assert solvent.shape == (nz, ny, nx)
    return {
        "lo": tuple(float(v) for v in lo), "hi": tuple(float(v) for v in hi), "dims": (nx, ny, nz),
        "conc": conc, "conc_uniform": np.zeros(D, dtype=np.float32), "solvent": solvent,
        "sigma_s": float(sigma_s), "sigma_a0": float(sigma_a0),
        "wall_mask": int(wall_mask), "wall_albedo": float(wall_albedo),
    }


def pencil_beam(origin, direction, lines_nm, power=None):
    lines_nm = list(lines_nm)
    return {"kind": "collimated", "origin": tuple(map(float, origin)), "eu": (0.0, 0.0, 0.0),
            "ev": (0.0, 0.0, 0.0), "dir": tuple(map(float, direction)), "lines_nm": lines_nm,
            "power": list(power) if power is not None else [1.0] * len(lines_nm)}


def rect_source(kind, origin, eu, ev, direction, lines_nm, power=None):
    lines_nm = list(lines_nm)
    return {"kind": kind, "origin": tuple(map(float, origin)), "eu": tuple(map(float, eu)),
            "ev": tuple(map(float, ev)), "dir": tuple(map(float, direction)), "lines_nm": lines_nm,
            "power": list(power) if power is not None else [1.0] * len(lines_nm)}


def no_sensor():
    return {"kind": "none", "width": 0, "height": 0, "origin": (0, 0, 0), "U": (0, 0, 0),
            "V": (0, 0, 0), "view": (0, 0, 0), "fov_y_deg": 0.0}


def ortho_sensor(width, height, origin, U, V, view):
    return {"kind": "ortho", "width": int(width), "height": int(height),
            "origin": tuple(map(float, origin)), "U": tuple(map(float, U)),
            "V": tuple(map(float, V)), "view": tuple(map(float, view)), "fov_y_deg": 0.0}


def pinhole_sensor(width, height, eye, right, up, forward, fov_y_deg):
    return {"kind": "pinhole", "width": int(width), "height": int(height),
            "origin": tuple(map(float, eye)), "U": tuple(map(float, right)),
            "V": tuple(map(float, up)), "view": tuple(map(float, forward)),
            "fov_y_deg": float(fov_y_deg)}


def params(n_paths, seed=0, n_rr=5, max_events=1_000_000, max_inelastic=-1, analog=0,
           max_steps=10_000_000):
    return {"n_paths": int(n_paths), "seed": int(seed), "n_rr": int(n_rr),
            "max_events": int(max_events), "max_inelastic": int(max_inelastic),
            "analog": int(analog), "max_steps": int(max_steps)}


# ------------------------------------------------------------------------------------------
# Workloads


def cfg1_homogeneous_cube(n_paths=100_000, film=64, seed=0):
    """1 cm cube, sigma_s 20 cm^-1, one dye: absorption Gauss(490, 15) with peak 2 cm^-1,
    emission Gauss(520, 20), QY 0.9, c = 1; pencil beam at 490 nm entering the centre of the
    +z face heading -z; 64x64 orthographic film of the +z face; RR after 5 events."""
    dyes = make_dyes([490.0], [15.0], [520.0], [20.0], eps=[2.0], qy=[0.9])
    return {
        "name": "cfg1_homogeneous_cube",
        "spectrum": spectrum(), "dyes": dyes,
        "medium": homogeneous_medium(1, conc=1.0, sigma_s=20.0),
        "sources": [pencil_beam((0.5, 0.5, 1.0), (0.0, 0.0, -1.0), [490.0])],
        "sensor": ortho_sensor(film, film, (0, 0, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1)),
        "params": params(n_paths, seed=seed, n_rr=5),
    }


def _place_spheres(rng, n, rmin, rmax, lo=0.0, hi=1.0, tries=10000):
    out = []
    for _ in range(tries):
        if len(out) == n:
            break
        r = rng.uniform(rmin, rmax)
        c = rng.uniform(lo + r, hi - r, size=3)
        if all(np.linalg.norm(c - c2) >= r + r2 + 0.01 for c2, r2 in out):
            out.append((c, r))
    if len(out) != n:
        raise RuntimeError("could not place spheres")
    return out


def voxel_centres(n, lo=0.0, hi=1.0):
    h = (hi - lo) / n
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * h


def cfg2_cornell_box(width=512, height=512, spp=16, grid=128, seed=0, n_paths=None,
                     wall_gloss=0.0, wall_exponent=0.0):
    """Cornell-box-style scene: a 1 cm box with Lambertian walls (rho 0.8) on all faces but the
    open front (-y); 4 non-overlapping dye spheres (radius 0.15-0.25 box), each filled with one
    Gaussian dye (emission peaks 450/520/600/680 nm, absorption peaks 30 nm lower, sigma 15/20 nm,
    QY U[0.3, 0.95], peak absorption 2 cm^-1 at c = 1) dissolved in a solvent with sigma_s 50
    cm^-1; the air between spheres is empty. A ceiling area light (Lambertian, facing down)
    emits 4 equal lines at the dyes' absorption peaks. A 512x512 pinhole camera (40 deg vertical
    FOV) looks into the box through the open front. Paths = pixels x spp."""
    rng = np.random.default_rng(seed)
    em_peaks = [450.0, 520.0, 600.0, 680.0]
    abs_peaks = [p - 30.0 for p in em_peaks]
    qy = rng.uniform(0.3, 0.95, size=4)
    dyes = make_dyes(abs_peaks, [15.0] * 4, em_peaks, [20.0] * 4, eps=[2.0] * 4, qy=qy)
    spheres = _place_spheres(rng, 4, 0.15, 0.25)
    xc = voxel_centres(grid)
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    conc = np.zeros((4, grid, grid, grid), dtype=np.float32)
    solvent = np.zeros((grid, grid, grid), dtype=np.uint8)
    for d, (c, r) in enumerate(spheres):
        inside = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 <= r * r
        conc[d][inside] = 1.0
        solvent[inside] = 1
    walls = 0b111111 & ~(1 << FACE_NY)
    med = grid_medium(conc, solvent, sigma_s=50.0, wall_mask=walls, wall_albedo=0.8)
    if wall_gloss > 0.0:   # the paper's glossy Cornell box (Sec. 5)
        med["wall_gloss"] = float(wall_gloss)
        med["wall_exponent"] = float(wall_exponent)
    light = rect_source("lambertian", (0.35, 0.35, 1.0), (0.3, 0.0, 0.0), (0.0, 0.3, 0.0),
                        (0.0, 0.0, -1.0), abs_peaks)
    cam = pinhole_sensor(width, height, eye=(0.5, -1.4, 0.5), right=(1, 0, 0), up=(0, 0, 1),
                         forward=(0, 1, 0), fov_y_deg=40.0)
    n = n_paths if n_paths is not None else width * height * spp
    return {
        "name": "cfg2_cornell_box", "spheres": [(tuple(c), float(r)) for c, r in spheres],
        "spectrum": spectrum(), "dyes": dyes, "medium": med, "sources": [light], "sensor": cam,
        "params": params(n, seed=seed, n_rr=5),
    }


def blob_field(rng, n, n_blobs, sigma_vox=(2.0, 8.0), amp=(0.5, 1.5)):
    """Sum of isotropic Gaussians on an n^3 voxel grid (z, y, x order), centres uniform in the
    grid, widths and amplitudes uniform; each blob is evaluated within +-3 sigma."""
    g = np.zeros((n, n, n), dtype=np.float32)
    centres = rng.uniform(0, n, size=(n_blobs, 3))
    sig = rng.uniform(sigma_vox[0], sigma_vox[1], size=n_blobs)
    amps = rng.uniform(amp[0], amp[1], size=n_blobs)
    idx = np.arange(n, dtype=np.float64) + 0.5
    for (cx, cy, cz), s, a in zip(centres, sig, amps):
        r = 3.0 * s
        x0, x1 = max(0, int(cx - r)), min(n, int(cx + r) + 1)
        y0, y1 = max(0, int(cy - r)), min(n, int(cy + r) + 1)
        z0, z1 = max(0, int(cz - r)), min(n, int(cz + r) + 1)
        gx = np.exp(-0.5 * ((idx[x0:x1] - cx) / s) ** 2)
        gy = np.exp(-0.5 * ((idx[y0:y1] - cy) / s) ** 2)
        gz = np.exp(-0.5 * ((idx[z0:z1] - cz) / s) ** 2)
        g[z0:z1, y0:y1, x0:x1] += (a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
                                   ).astype(np.float32)
    return g


def cfg3_batched_media(n_media=256, seed=0, path_scale=1.0, max_edge=128, min_edge=16,
                       sigma_t_ref=40.0):
    """256 independent 1 cm cubes. Per medium: grid edge n ~ U{16..128}, 1-3 Gaussian dyes,
    albedo ~ U[0.5, 0.999] at the source wavelength, half homogeneous (constant grids) and half
    blobby, paths log-uniform in [1e4, 1e6] (times path_scale). A pencil beam at the first dye's
    absorption peak enters the -z face centre heading +z. Dye absorption is scaled so that
    sum_d eps_d a_d(lambda_src) mean(c_d) = (1 - albedo) sigma_t_ref, sigma_s = albedo sigma_t_ref."""
    rng = np.random.default_rng(seed)
    media = []
    for m in range(n_media):
        n = int(rng.integers(min_edge, max_edge + 1))
        D = int(rng.integers(1, 4))
        albedo = float(rng.uniform(0.5, 0.999))
        hetero = bool(rng.random() < 0.5)
        n_paths = int(round(10 ** rng.uniform(4.0, 6.0) * path_scale))
        abs_p = rng.uniform(420.0, 620.0, size=D)
        abs_p[1:] = abs_p[0] + rng.uniform(-25.0, 25.0, size=D - 1)
        em_p = abs_p + rng.uniform(20.0, 60.0, size=D)
        qy = rng.uniform(0.3, 0.95, size=D)
        a_sig = rng.uniform(12.0, 25.0, size=D)
        e_sig = rng.uniform(15.0, 30.0, size=D)
        if hetero:
            conc = np.stack([blob_field(rng, n, 8, (n / 16, n / 6)) for _ in range(D)])
            conc /= conc.reshape(D, -1).mean(axis=1)[:, None, None, None]
        else:
            conc = np.ones((D, n, n, n), dtype=np.float32)
        lam_src = float(abs_p[0])
        dy0 = make_dyes(abs_p, a_sig, em_p, e_sig, eps=np.ones(D), qy=qy)
        src_bin = int(np.clip(math.ceil((lam_src - LAMBDA0) / DLAMBDA - 0.5), 0, N_BINS - 1))
        a_src = dy0["abs_shape"][:, src_bin].astype(np.float64)
        mean_c = conc.reshape(D, -1).mean(axis=1).astype(np.float64)
        eps = (1.0 - albedo) * sigma_t_ref / float(np.sum(a_src * mean_c))
        dyes = make_dyes(abs_p, a_sig, em_p, e_sig, eps=np.full(D, eps), qy=qy)
        med = grid_medium(conc.astype(np.float32), None, sigma_s=albedo * sigma_t_ref)
        media.append({
            "name": f"cfg3_medium_{m}", "spectrum": spectrum(), "dyes": dyes, "medium": med,
            "sources": [pencil_beam((0.5, 0.5, 0.0), (0.0, 0.0, 1.0), [lam_src])],
            "sensor": no_sensor(), "params": params(n_paths, seed=seed, n_rr=5),
            "albedo": albedo, "edge": n, "hetero": hetero,
        })
    return media


def cfg4_adjoint(field_seed=0, grid=64, width=256, height=256, spp=32, seed=0, n_paths=None,
                 sigma_s=30.0):
    """Adjoint scene: 64^3 grid, 2 blobby dyes (field_seed 0 = current, 1 = target),
    sigma_s 30 cm^-1, a uniform collimated beam over the whole -z face heading +z with two lines at
    the dyes' absorption peaks, orthographic 256x256 film of the +z face, 32 spp."""
    rng = np.random.default_rng(1000 + field_seed)
    conc = np.stack([blob_field(rng, grid, 24, (3.0, 8.0)) for _ in range(2)])
    conc /= conc.reshape(2, -1).mean(axis=1)[:, None, None, None]
    dyes = make_dyes([470.0, 560.0], [15.0, 15.0], [520.0, 610.0], [20.0, 20.0], eps=[2.0, 2.0],
                     qy=[0.8, 0.6])
    med = grid_medium(conc.astype(np.float32), None, sigma_s=sigma_s)
    src = rect_source("collimated", (0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0),
                      (0.0, 0.0, 1.0), [470.0, 560.0])
    cam = ortho_sensor(width, height, (0, 0, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1))
    n = n_paths if n_paths is not None else width * height * spp
    return {"name": f"cfg4_adjoint_field{field_seed}", "spectrum": spectrum(), "dyes": dyes,
            "medium": med, "sources": [src], "sensor": cam, "params": params(n, seed=seed)}


def cfg5_light_sheet(grid=256, width=1024, height=1024, spp=64, seed=0, n_paths=None,
                     n_blobs=500, albedo=0.999, sigma_t_ref=63.0):
    """Light-sheet scene: 256^3 grid, 4 dyes each a sum of 500 Gaussian blobs (sigma 2-8 voxels),
    albedo 0.999 at 490 nm (about 1000 events per path). The sheet (488 nm, snapped to the 490 nm
    bin) enters the -x face and propagates along +x, 0.05 cm thick about z = 0.5 and spanning y;
    a 1024x1024 orthographic camera views the sheet face-on from +z (90 degrees to the
    illumination axis), 64 spp."""
    rng = np.random.default_rng(seed)
    conc = np.stack([blob_field(rng, grid, n_blobs, (2.0, 8.0)) for _ in range(4)])
    conc /= conc.reshape(4, -1).mean(axis=1)[:, None, None, None]
    abs_p = [480.0, 495.0, 510.0, 530.0]
    em_p = [520.0, 560.0, 600.0, 650.0]
    dy0 = make_dyes(abs_p, [15.0] * 4, em_p, [20.0] * 4, eps=np.ones(4), qy=[0.9, 0.7, 0.6, 0.5])
    src_bin = int(math.ceil((488.0 - LAMBDA0) / DLAMBDA - 0.5))
    a_src = dy0["abs_shape"][:, src_bin].astype(np.float64)
    eps = (1.0 - albedo) * sigma_t_ref / float(np.sum(a_src * 1.0))
    dyes = make_dyes(abs_p, [15.0] * 4, em_p, [20.0] * 4, eps=np.full(4, eps),
                     qy=[0.9, 0.7, 0.6, 0.5])
    med = grid_medium(conc.astype(np.float32), None, sigma_s=albedo * sigma_t_ref)
    src = rect_source("collimated", (0.0, 0.0, 0.475), (0.0, 1.0, 0.0), (0.0, 0.0, 0.05),
                      (1.0, 0.0, 0.0), [488.0])
    cam = ortho_sensor(width, height, (0, 0, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1))
    n = n_paths if n_paths is not None else width * height * spp
    return {"name": "cfg5_light_sheet", "spectrum": spectrum(), "dyes": dyes, "medium": med,
            "sources": [src], "sensor": cam, "params": params(n, seed=seed)}


def paper_mode_scene(n=16, width=8, spp=1000, seed=7, sigma_s=3.0):
    """Workload of the paper's own (camera-side) estimator: two blobby dyes (absorption 470/560
    nm, emission 520/610 nm, sigma 20/25 nm) dissolved in a scattering solvent (sigma_s everywhere,
    so sigma_t > 0 wherever a dye is), Lambertian walls (rho 0.7) on the +-x faces, a uniform
    collimated beam over the -z face carrying the two absorption lines, and a pinhole camera
    (50 deg) looking in through the open -y face. Paths = pixels x spp."""
    rng = np.random.default_rng(seed)
    conc = np.stack([blob_field(rng, n, 6, (1.5 * n / 16, 3.0 * n / 16)) for _ in range(2)])
    conc /= conc.reshape(2, -1).mean(axis=1)[:, None, None, None]
    dyes = make_dyes([470.0, 560.0], [20.0, 20.0], [520.0, 610.0], [25.0, 25.0], eps=[3.0, 2.0],
                     qy=[0.8, 0.6])
    walls = (1 << FACE_NX) | (1 << FACE_PX)
    med = grid_medium(conc.astype(np.float32), None, sigma_s=sigma_s, wall_mask=walls,
                      wall_albedo=0.7)
    beam = rect_source("collimated", (0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0),
                       (0.0, 0.0, 1.0), [470.0, 560.0])
    cam = pinhole_sensor(width, width, eye=(0.5, -1.0, 0.5), right=(1, 0, 0), up=(0, 0, 1),
                         forward=(0, 1, 0), fov_y_deg=50.0)
    return {"name": "paper_mode_scene", "spectrum": spectrum(), "dyes": dyes, "medium": med,
            "sources": [beam], "sensor": cam,
            "params": params(width * width * spp, seed=2)}


def vial_scene(conc_gpl=1.0, ior=1.33, width=64, height=64, spp=16, seed=0, n_paths=None,
               sigma_s=20.0, grid=None):
    """The paper's dye vials (Sec. 5: AF488 solutions at 0.1, 1 and 10 g/L lit at 495 nm), as a
    1 cm cuvette of solution with refractive index `ior` (water 1.33) whose six faces are smooth
    dielectric interfaces to the air: one Gaussian dye (absorption 495/15 nm, emission 520/20 nm,
    QY 0.9, peak absorption 1.5 cm^-1 per g/L) at `conc_gpl` in a scattering solvent (sigma_s),
    a collimated 1 mm beam at 495 nm entering the -x face at the centre, and an orthographic
    camera looking at the front (-y) face head-on (radiance travelling along -y). With `grid` the
    dye fills a centred cylinder (the vial) of radius 0.35 cm along z on an n^3 grid instead of
    the whole cuvette."""
    dyes = make_dyes([495.0], [15.0], [520.0], [20.0], eps=[1.5], qy=[0.9])
    if grid:
        xc = voxel_centres(grid)
        Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
        inside = (X - 0.5) ** 2 + (Y - 0.5) ** 2 <= 0.35 ** 2
        conc = (inside * conc_gpl).astype(np.float32)[None]
        med = grid_medium(conc, inside.astype(np.uint8), sigma_s=sigma_s)
    else:
        med = homogeneous_medium(1, conc=conc_gpl, sigma_s=sigma_s)
    med["ior"] = float(ior)
    beam = rect_source("collimated", (0.0, 0.45, 0.45), (0.0, 0.1, 0.0), (0.0, 0.0, 0.1),
                       (1.0, 0.0, 0.0), [495.0])
    cam = ortho_sensor(width, height, (0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 0.0, 1.0),
                       (0.0, -1.0, 0.0))
    n = n_paths if n_paths is not None else width * height * spp
    return {"name": "vial", "spectrum": spectrum(), "dyes": dyes, "medium": med,
            "sources": [beam], "sensor": cam, "params": params(n, seed=seed, n_rr=5)}
