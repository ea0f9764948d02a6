"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage it checks. Tolerances are 3 standard errors for single quantities
(binomial or batch-means SE), and Wilson-Hilferty chi-square bounds for histograms. Seeds are
fixed, so every outcome is deterministic.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg
from tests.stats import batch_mean_se, binomial_se, chi2_counts, chi2_ok

B = sg.N_BINS


def bin_of(lam):
    return int(math.ceil((lam - sg.LAMBDA0) / sg.DLAMBDA - 0.5))


def slab_scene(n_paths, sigma_s=0.0, sigma_a0=0.0, dyes=None, conc=1.0, beam_nm=490.0,
               lo=(0, 0, 0), hi=(1, 1, 1), sensor=None, beam_origin=None, beam_dir=(0, 0, -1)):
    if dyes is None:
        dyes = sg.make_dyes([490.0], [15.0], [620.0], [15.0], eps=[0.0], qy=[0.0])
    D = dyes["eps"].shape[0]
    if beam_origin is None:
        beam_origin = (0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), hi[2])
    return {
        "spectrum": sg.spectrum(), "dyes": dyes,
        "medium": sg.homogeneous_medium(D, conc=conc, sigma_s=sigma_s, sigma_a0=sigma_a0, lo=lo,
                                        hi=hi),
        "sources": [sg.pencil_beam(beam_origin, beam_dir, [beam_nm])],
        "sensor": sensor or sg.no_sensor(),
        "params": sg.params(n_paths, seed=7),
    }


def batched(scene, K, n_per, **kw):
    outs = [oracle.render(scene, n_paths=n_per, path_offset=k * n_per, **kw) for k in range(K)]
    return outs


# ------------------------------------------------------------------------------------------
# RNG: Philox4x32-10 (Salmon et al. 2011) -- statistical properties of the generator


def test_philox_uniformity_and_independence():
    n = 1 << 18
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    out = oracle.philox(0, 0, ctr)
    u = (out >> 8).astype(np.float64) / 2.0 ** 24
    # each output word uniform: 64-bin chi-square
    for j in range(4):
        h = np.bincount((u[:, j] * 64).astype(int), minlength=64)
        chi2, dof = chi2_counts(h, np.full(64, 1 / 64))
        assert chi2_ok(chi2, dof), (j, chi2)
    # words within a block and consecutive counters uncorrelated
    c = np.corrcoef(u.T)
    assert np.abs(c - np.eye(4)).max() < 4.0 / math.sqrt(n) * 1.5
    lag = np.corrcoef(u[:-1, 0], u[1:, 0])[0, 1]
    assert abs(lag) < 4.0 / math.sqrt(n)
    # bit balance of the raw 32-bit outputs
    bits = np.unpackbits(out.view(np.uint8)).reshape(n, 128).mean(axis=0)
    assert np.abs(bits - 0.5).max() < 5 * 0.5 / math.sqrt(n)


def test_philox_avalanche_on_counter_key_and_slot():
    rng = np.random.default_rng(3)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    base = oracle.philox(11, 5, ctr)
    for word in range(4):
        flipped = ctr.copy()
        flipped[:, word] ^= np.uint32(1 << int(rng.integers(0, 32)))
        diff = oracle.philox(11, 5, flipped) ^ base
        frac = np.unpackbits(diff.view(np.uint8)).mean()
        assert abs(frac - 0.5) < 0.01, (word, frac)
    other_key = oracle.philox(12, 5, ctr) ^ base
    assert abs(np.unpackbits(other_key.view(np.uint8)).mean() - 0.5) < 0.01
    other_med = oracle.philox(11, 6, ctr) ^ base
    assert abs(np.unpackbits(other_med.view(np.uint8)).mean() - 0.5) < 0.01


# ------------------------------------------------------------------------------------------
# Eq. 10: emission wavelength drawn from the normalised emission spectrum


def test_emission_sampling_matches_normalised_spectrum():
    dyes = sg.make_dyes([490.0, 400.0], [15.0, 10.0], [520.0, 610.0], [20.0, 35.0],
                        eps=[1.0, 1.0], qy=[1.0, 1.0])
    sc = slab_scene(1, dyes=dyes)
    rng = np.random.default_rng(0)
    u = (rng.integers(0, 2 ** 24, size=400_000) / 2.0 ** 24)
    for d in range(2):
        bins = oracle.sample_emission(sc, d, u)
        assert bins.min() >= 0 and bins.max() < B
        pmf = dyes["emit_spec"][d].astype(np.float64)
        pmf /= pmf.sum()
        chi2, dof = chi2_counts(np.bincount(bins, minlength=B), pmf)
        assert chi2_ok(chi2, dof), (d, chi2, dof)
        assert abs(bins.mean() - (pmf * np.arange(B)).sum()) < 0.05


def test_emission_sampling_single_line_and_extremes():
    em = np.zeros((1, B), np.float32)
    em[0, 37] = 3.0
    dyes = {"abs_shape": sg.gaussian_band(490, 15)[None], "emit_spec": em,
            "eps": np.ones(1, np.float32), "qy": np.ones(1, np.float32)}
    sc = slab_scene(1, dyes=dyes)
    u = np.array([0.0, 0.25, 0.5, 1.0 - 2.0 ** -24])
    assert (oracle.sample_emission(sc, 0, u) == 37).all()
    # two equal lines: u below one half picks the first, from one half on the second
    em[0, 10] = 3.0
    dyes["emit_spec"] = em
    sc = slab_scene(1, dyes=dyes)
    got = oracle.sample_emission(sc, 0, np.array([0.0, 0.5 - 2 ** -24, 0.5, 0.99]))
    assert list(got) == [10, 10, 37, 37]


# ------------------------------------------------------------------------------------------
# Sec. 2.1: isotropic emission and scattering; Lambertian walls and lights


def test_isotropic_direction_moments():
    rng = np.random.default_rng(1)
    n = 400_000
    w = oracle.iso_dir(rng.random(n), rng.random(n))
    assert np.allclose(np.linalg.norm(w, axis=1), 1.0, atol=1e-12)
    se = math.sqrt(1 / 3 / n)
    assert np.abs(w.mean(axis=0)).max() < 4 * se
    m2 = (w[:, :, None] * w[:, None, :]).mean(axis=0)
    assert np.abs(m2 - np.eye(3) / 3).max() < 4 * math.sqrt(0.09 / n)


@pytest.mark.parametrize("axis,sign", [(0, 1.0), (1, -1.0), (2, -1.0)])
def test_cosine_direction_moments(axis, sign):
    rng = np.random.default_rng(2)
    n = 400_000
    w = oracle.cosine_dir(rng.random(n), rng.random(n), axis, sign)
    assert np.allclose(np.linalg.norm(w, axis=1), 1.0, atol=1e-12)
    c = sign * w[:, axis]
    assert c.min() >= 0.0
    # cosine-weighted hemisphere: E[cos] = 2/3, E[cos^2] = 1/2, tangents mean zero
    assert abs(c.mean() - 2 / 3) < 4 * math.sqrt(1 / 18 / n)
    assert abs((c ** 2).mean() - 0.5) < 4 * math.sqrt(1 / 12 / n)
    t = [k for k in range(3) if k != axis]
    assert np.abs(w[:, t].mean(axis=0)).max() < 4 * math.sqrt(0.25 / n)


# ------------------------------------------------------------------------------------------
# Eq. 6 (Beer-Lambert transmittance): exact optical depth over piecewise-constant voxels


def ramp_grid_scene(n, axis, sigma_per_unit=1.0):
    """Single dye whose concentration equals (voxel index along `axis`) + 1."""
    idx = np.arange(n, dtype=np.float32) + 1.0
    shape = [1, 1, 1]
    shape[2 - axis] = n
    conc = np.broadcast_to(idx.reshape(shape), (n, n, n)).astype(np.float32)[None].copy()
    dyes = sg.make_dyes([490.0], [15.0], [620.0], [15.0], eps=[sigma_per_unit], qy=[0.0])
    return {"spectrum": sg.spectrum(), "dyes": dyes, "medium": sg.grid_medium(conc),
            "sources": [sg.pencil_beam((0.5, 0.5, 1), (0, 0, -1), [490.0])],
            "sensor": sg.no_sensor(), "params": sg.params(1)}


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_optical_depth_axis_and_oblique(axis):
    n = 8
    sc = ramp_grid_scene(n, axis, 2.0)
    b = bin_of(490)
    h = 1.0 / n
    # ray along the ramp axis through the whole cube: sum of the ramp times the voxel length
    x0 = np.full(3, 0.37)
    x0[axis] = 0.0
    w = np.zeros(3)
    w[axis] = 1.0
    exact = 2.0 * h * np.sum(np.arange(n) + 1.0)
    assert abs(oracle.optical_depth(sc, x0, w, 1.0, b) - exact) < 1e-12 * exact
    # ray perpendicular to the ramp: constant voxel value times the length
    w2 = np.zeros(3)
    w2[(axis + 1) % 3] = 1.0
    x1 = np.full(3, 0.0)
    x1[axis] = 0.3  # voxel index 2 -> value 3
    x1[(axis + 2) % 3] = 0.6
    assert abs(oracle.optical_depth(sc, x1, w2, 1.0, b) - 2.0 * 3.0) < 1e-12
    # oblique ray: each slab along `axis` is crossed over a length h / |w_axis|
    w3 = np.array([0.6, 0.48, 0.64])
    w3 /= np.linalg.norm(w3)
    L = 1.0 / w3.max()  # stays inside the cube from the origin corner
    tau = oracle.optical_depth(sc, np.zeros(3), w3, L, b)
    # slab k along `axis` covers parameter range [k h / w_a, (k+1) h / w_a] clipped to [0, L]
    wa = w3[axis]
    exact = 0.0
    for k in range(n):
        a0, a1 = k * h / wa, (k + 1) * h / wa
        seg = max(0.0, min(a1, L) - max(a0, 0.0))
        exact += 2.0 * (k + 1) * seg
    assert abs(tau - exact) < 1e-9


def test_beer_lambert_nonscattering_slab():
    """Eq. 6: a non-scattering absorber transmits exp(-sigma_a L) of a normal pencil beam."""
    n = 200_000
    for sa0, dye_eps in ((1.3, 0.0), (0.0, 0.9)):
        dyes = sg.make_dyes([490.0], [15.0], [620.0], [15.0], eps=[dye_eps], qy=[0.0])
        sc = slab_scene(n, sigma_a0=sa0, dyes=dyes)
        for analog in (0, 1):
            r = oracle.render(sc, analog=analog)
            T = r["face"][:, sg.FACE_NZ, :].sum()
            exact = math.exp(-(sa0 + dye_eps))
            assert abs(T - exact) <= 3 * binomial_se(exact, n), (sa0, dye_eps, analog, T, exact)
            assert r["counters"]["scatters"] == 0
            # every absorbed photon is in the absorbed tally
            assert abs(r["absorbed"].sum() + r["face"].sum() - 1.0) < 1e-12


def test_uncollided_transmission_heterogeneous_grid():
    """Delta tracking (free flights against the majorant) must reproduce the exact uncollided
    transmission exp(-int sigma_t) of Eq. 6 through a heterogeneous grid."""
    rng = np.random.default_rng(5)
    n = 6
    conc = rng.uniform(0.0, 2.0, size=(2, n, n, n)).astype(np.float32)
    solvent = (rng.random((n, n, n)) < 0.7).astype(np.uint8)
    dyes = sg.make_dyes([490.0, 500.0], [15.0, 30.0], [620.0, 650.0], [15.0, 15.0],
                        eps=[0.4, 0.3], qy=[0.5, 0.5])
    med = sg.grid_medium(conc, solvent, sigma_s=0.8)
    x, y = 0.41, 0.77
    sc = {"spectrum": sg.spectrum(), "dyes": dyes, "medium": med,
          "sources": [sg.pencil_beam((x, y, 1.0), (0, 0, -1), [490.0])],
          "sensor": sg.no_sensor(), "params": sg.params(200_000, seed=3)}
    N = 200_000
    r = oracle.render(sc, max_events=0)  # the first real collision ends the path
    T = r["face"][:, sg.FACE_NZ, :].sum()
    b = bin_of(490)
    # exact: sum over the beam's voxel column of sigma_t times the voxel height
    ix, iy = int(x * n), int(y * n)
    a = dyes["abs_shape"][:, b].astype(np.float64) * dyes["eps"].astype(np.float64)
    col = (solvent[:, iy, ix] * 0.8 + a[0] * conc[0, :, iy, ix] + a[1] * conc[1, :, iy, ix])
    exact = math.exp(-col.sum() / n)
    assert abs(T - exact) <= 3 * binomial_se(exact, N), (T, exact)
    assert abs(oracle.optical_depth(sc, np.array([x, y, 1.0]), np.array([0, 0, -1.0]), 1.0, b)
               - col.sum() / n) < 1e-12
    assert r["counters"]["nulls"] > 0
    assert r["counters"]["majorant_violations"] == 0


# ------------------------------------------------------------------------------------------
# Photon bookkeeping and QY (Sec. 4.1)


def test_conservation_analog_integer_identity():
    sc = sg.cfg1_homogeneous_cube(n_paths=50_000)
    sc["medium"]["sigma_a0"] = 0.3
    r = oracle.render(sc, analog=1)
    c = r["counters"]
    ends = (c["escapes"] + c["absorbed_dead"] + c["rr_kills"] + c["cap_hits"] + c["step_budget"]
            + c["vf_rejected"])
    assert ends == c["paths"] == 50_000
    assert c["rr_kills"] == 0  # analog weights stay 1, so roulette never kills
    assert c["events"] == c["scatters"] + c["dye_absorptions"] + (
        c["absorbed_dead"] - (c["dye_absorptions"] - c["emissions"]))
    # escaped photon count equals the summed face tally (unit weights)
    assert abs(r["face"].sum() * 50_000 - c["escapes"]) < 1e-6


def test_conservation_scattering_only_is_exact():
    sc = slab_scene(20_000, sigma_s=15.0)
    for analog in (0, 1):
        r = oracle.render(sc, analog=analog)
        assert abs(r["face"].sum() - 1.0) < 1e-12
        assert r["counters"]["escapes"] == 20_000


def test_weighted_mode_expected_conservation():
    """Weighted mode: escaped power = 1 - background absorbed - sum_d (1 - QY_d) absorbed_d,
    in expectation (roulette is unbiased)."""
    sc = sg.cfg1_homogeneous_cube()
    sc["medium"]["sigma_a0"] = 0.2
    outs = batched(sc, 16, 8000)
    lhs = np.array([o["face"].sum() for o in outs])
    rhs = np.array([1.0 - o["absorbed"][1].sum() - (1 - 0.9) * o["absorbed"][0].sum()
                    for o in outs])
    m, se = batch_mean_se(lhs - rhs)
    assert abs(m) <= 3 * se + 1e-12, (m, se)


def test_quantum_yield_weighted_exact_and_analog_binomial():
    dyes = sg.make_dyes([490.0, 500.0], [15.0, 15.0], [520.0, 560.0], [20.0, 20.0],
                        eps=[2.0, 1.0], qy=[0.9, 0.35])
    sc = slab_scene(60_000, sigma_s=10.0, dyes=dyes)
    r = oracle.render(sc, analog=0)
    for d, qy in enumerate((0.9, 0.35)):
        q32 = float(np.float32(qy))
        assert abs(r["emitted"][d].sum() - q32 * r["absorbed"][d].sum()) < 1e-12
    r = oracle.render(sc, analog=1)
    c = r["counters"]
    # two dyes: emissions ~ sum of binomials; check the combined expectation with its SD
    em = r["emitted"].sum(axis=1) * 60_000
    ab = r["absorbed"][:2].sum(axis=1) * 60_000
    for d, qy in enumerate((0.9, 0.35)):
        q = float(np.float32(qy))
        assert abs(em[d] - q * ab[d]) <= 3 * math.sqrt(ab[d] * q * (1 - q)), (d, em[d], ab[d])
    assert c["emissions"] == int(round(em.sum()))


def test_event_choice_in_proportion_to_coefficients():
    """Sec. 4.1: a collision is with dye d with probability sigma_a,d / sigma_t."""
    dyes = sg.make_dyes([480.0, 520.0], [15.0, 15.0], [640.0, 700.0], [10.0, 10.0],
                        eps=[0.3, 0.5], qy=[0.0, 0.0])
    sc = slab_scene(200_000, sigma_s=0.4, sigma_a0=0.1, dyes=dyes)
    r = oracle.render(sc, analog=1, max_events=1)
    c = r["counters"]
    b = bin_of(490)
    s = np.array([0.4, 0.3 * dyes["abs_shape"][0, b], 0.5 * dyes["abs_shape"][1, b], 0.1],
                 dtype=np.float64)
    p = s / s.sum()
    n_ev = c["events"]
    got = np.array([c["scatters"], r["absorbed"][0].sum() * 200_000,
                    r["absorbed"][1].sum() * 200_000, r["absorbed"][2].sum() * 200_000])
    chi2, dof = chi2_counts(np.round(got), p)
    assert chi2_ok(chi2, dof), (got / n_ev, p)


def test_single_inelastic_mode():
    """Sec. 4.1 / Eq. 9: with at most one inelastic event, a second dye absorption ends the path
    (V_f = 0); with zero allowed, nothing is re-emitted."""
    sc = sg.cfg1_homogeneous_cube(n_paths=20_000)
    r0 = oracle.render(sc, max_inelastic=0)
    assert r0["emitted"].sum() == 0.0
    assert r0["counters"]["vf_rejected"] == r0["counters"]["dye_absorptions"]
    r1 = oracle.render(sc, max_inelastic=1)
    c = r1["counters"]
    assert c["emissions"] + c["vf_rejected"] == c["dye_absorptions"]
    assert c["vf_rejected"] > 0
    assert r1["face"][1].sum() > 0


# ------------------------------------------------------------------------------------------
# Paper validations (Sec. 6): emission profile of a thin dye, and scaling with f_x(lambda_x)


def _solid_angle_triangle(p, a, b, c):
    ra, rb, rc = a - p, b - p, c - p
    la, lb, lc = np.linalg.norm(ra), np.linalg.norm(rb), np.linalg.norm(rc)
    num = abs(np.dot(ra, np.cross(rb, rc)))
    den = la * lb * lc + np.dot(ra, rb) * lc + np.dot(ra, rc) * lb + np.dot(rb, rc) * la
    return 2.0 * math.atan2(num, den)


def face_solid_angles(p):
    """Solid angle of each unit-cube face (-x,+x,-y,+y,-z,+z) from an interior point
    (Van Oosterom-Strackee triangle formula, two triangles per face)."""
    out = []
    for axis in range(3):
        for side in (0.0, 1.0):
            u, v = (axis + 1) % 3, (axis + 2) % 3
            corners = []
            for cu, cv in ((0, 0), (1, 0), (1, 1), (0, 1)):
                q = np.zeros(3)
                q[axis], q[u], q[v] = side, cu, cv
                corners.append(q)
            out.append(_solid_angle_triangle(p, corners[0], corners[1], corners[2])
                       + _solid_angle_triangle(p, corners[0], corners[2], corners[3]))
    return np.array(out)


def thin_dye_scene(n_paths, eps, lam_x=450.0, qy=0.8):
    # absorption band far below the emission band, so emitted light is never re-absorbed
    dyes = sg.make_dyes([450.0], [10.0], [620.0], [18.0], eps=[eps], qy=[qy])
    return slab_scene(n_paths, dyes=dyes, beam_nm=lam_x)


def test_thin_dye_reproduces_emission_spectrum():
    """Validation 1 (Sec. 6): the normalised emission SPD of an optically thin dye matches the
    dye's emission spectrum."""
    n = 400_000
    sc = thin_dye_scene(n, eps=0.05, qy=1.0)
    r = oracle.render(sc, analog=1)
    spd = r["face"][1].sum(axis=0) * n  # fluoresced photons per bin, all faces
    pmf = sc["dyes"]["emit_spec"][0].astype(np.float64)
    pmf /= pmf.sum()
    chi2, dof = chi2_counts(np.round(spd), pmf)
    assert chi2_ok(chi2, dof), (chi2, dof)
    assert r["face"][0, :, :bin_of(560)].sum() > 0.9  # the rest leaves at the excitation line


def test_slab_fluorescence_yield_and_face_split():
    """Validation 2 (Sec. 6) in closed form: a non-scattering cube lit by a pencil beam at
    lambda_x re-emits QY (1 - exp(-sigma_a(lambda_x) L)); each face receives the absorption
    density times its solid angle over 4 pi."""
    n = 300_000
    qy = 0.8
    for lam_x in (440.0, 450.0, 470.0):
        sc = thin_dye_scene(n, eps=1.5, lam_x=lam_x, qy=qy)
        r = oracle.render(sc)
        sa = 1.5 * float(sc["dyes"]["abs_shape"][0, bin_of(lam_x)])
        q = float(np.float32(qy))
        total = r["face"][1].sum()
        p_abs = 1.0 - math.exp(-sa)
        assert abs(total - q * p_abs) <= 3 * q * binomial_se(p_abs, n), (lam_x, total)
        # per-face split: integrate the absorption density along the beam (depth s from +z)
        s = (np.arange(4000) + 0.5) / 4000
        dens = sa * np.exp(-sa * s) / 4000
        frac = np.zeros(6)
        for si, di in zip(s, dens):
            frac += di * face_solid_angles(np.array([0.5, 0.5, 1.0 - si])) / (4 * math.pi)
        got = r["face"][1].sum(axis=1)
        for f in range(6):
            p = frac[f] / p_abs
            se = q * math.sqrt(p_abs * p * (1 - p_abs * p) / n)
            assert abs(got[f] - q * frac[f]) <= 3 * se + 1e-9, (lam_x, f, got[f], q * frac[f])


def test_face_solid_angles_sum_to_sphere():
    for p in ([0.5, 0.5, 0.5], [0.1, 0.8, 0.3], [0.5, 0.5, 0.999]):
        assert abs(face_solid_angles(np.array(p)).sum() - 4 * math.pi) < 1e-9


# ------------------------------------------------------------------------------------------
# Multiple scattering: Chandrasekhar's plane albedo for an isotropic half-space


def chandrasekhar_H(albedo, n=64):
    x, wq = np.polynomial.legendre.leggauss(n)
    mu = 0.5 * (x + 1)
    w = 0.5 * wq
    H = np.ones(n)
    for _ in range(2000):
        Hn = 1.0 / (math.sqrt(1 - albedo) + 0.5 * albedo *
                    (w * mu * H / (mu[:, None] + mu[None, :])).sum(axis=1))
        if np.abs(Hn - H).max() < 1e-14:
            H = Hn
            break
        H = Hn

    def at(m):
        return 1.0 / (math.sqrt(1 - albedo) + 0.5 * albedo * (w * mu * H / (m + mu)).sum())
    return mu, w, H, at


def test_chandrasekhar_h_zeroth_moment_identity():
    for a in (0.5, 0.8, 0.95):
        mu, w, H, _ = chandrasekhar_H(a)
        assert abs(0.5 * a * (w * H).sum() - (1 - math.sqrt(1 - a))) < 1e-10


def test_half_space_plane_albedo():
    """Isotropic half-space, albedo a, normal incidence: reflectance 1 - H(1) sqrt(1 - a)."""
    n = 200_000
    for a in (0.6, 0.9):
        st = 10.0
        sc = slab_scene(n, sigma_s=a * st, sigma_a0=(1 - a) * st, lo=(-60, -60, 0),
                        hi=(60, 60, 12))
        r = oracle.render(sc, analog=1)
        R = r["face"][:, sg.FACE_PZ, :].sum()
        exact = 1.0 - chandrasekhar_H(a)[3](1.0) * math.sqrt(1 - a)
        assert abs(R - exact) <= 3 * binomial_se(exact, n), (a, R, exact)
        side = r["face"].sum() - R
        assert side < 1e-4


# ------------------------------------------------------------------------------------------
# Sensor connections (Eq. 3-6)


def test_emitter_line_choice_in_proportion_to_power():
    dyes = sg.make_dyes([490.0], [15.0], [620.0], [15.0], eps=[0.0], qy=[0.0])
    sc = slab_scene(100_000, dyes=dyes)
    sc["sources"] = [sg.pencil_beam((0.5, 0.5, 1.0), (0, 0, -1), [450.0, 600.0], [1.0, 3.0])]
    r = oracle.render(sc)
    f = r["face"][0, sg.FACE_NZ]
    assert abs(f[bin_of(600)] - 0.75) <= 3 * binomial_se(0.75, 100_000)
    assert abs(f.sum() - 1.0) < 1e-12


def test_ortho_single_scatter_and_emission_closed_form():
    """A pencil beam into a homogeneous cube, first collision only (max_events=1), ortho film of
    the entry face: film[centre, lambda_x] = (sigma_s/4pi A_pix) int e^{-2 sigma_t s} ds and
    film[centre, lambda'] = (QY p(lambda') sigma_a/4pi A_pix) int e^{-(sigma_t + sigma_t') s} ds."""
    W = 16
    sensor = sg.ortho_sensor(W, W, (0, 0, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1))
    dyes = sg.make_dyes([490.0], [15.0], [520.0], [20.0], eps=[2.0], qy=[0.9])
    sc = slab_scene(20_000, sigma_s=3.0, dyes=dyes, sensor=sensor)
    sc["sources"] = [sg.pencil_beam((0.53, 0.53, 1.0), (0, 0, -1), [490.0])]
    outs = batched(sc, 16, 20_000, max_events=1)
    films = np.stack([o["film"] for o in outs])
    m, se = batch_mean_se(films)
    A = 1.0 / (W * W)
    px = int(0.53 * W)
    bx = bin_of(490)
    a = dyes["abs_shape"][0].astype(np.float64) * 2.0
    st = 3.0 + a
    pmf = dyes["emit_spec"][0].astype(np.float64)
    pmf /= pmf.sum()
    q = float(np.float32(0.9))
    for b in range(B):
        exp_v = 0.0
        if b == bx:
            exp_v += 3.0 * (1 - math.exp(-2 * st[bx])) / (2 * st[bx])
        exp_v += q * pmf[b] * a[bx] * (1 - math.exp(-(st[bx] + st[b]))) / (st[bx] + st[b])
        exp_v /= 4 * math.pi * A
        got = m[px, px, b]
        # a bin may hold no sample at all: allow three single-sample contributions on top
        one = 1.0 / (4 * math.pi * A) / (16 * 20_000)
        assert abs(got - exp_v) <= 3 * se[px, px, b] + 3 * one, (b, got, exp_v)
    # nothing lands outside the beam's pixel
    mask = np.ones((W, W), bool)
    mask[px, px] = False
    assert m[mask].sum() == 0.0


def test_pinhole_single_scatter_quadrature():
    """Pinhole importance 1/(A_pix r^2 cos^3): summed over the film times A_pix, the first-collision
    image of a pencil beam equals int sigma_s e^{-sigma_t s} T(s)/(4 pi r^2 cos^3) ds."""
    W = 32
    eye = np.array([0.5, -2.0, 0.5])
    sensor = sg.pinhole_sensor(W, W, eye, (1, 0, 0), (0, 0, 1), (0, 1, 0), 45.0)
    sc = slab_scene(40_000, sigma_s=2.0, sensor=sensor)
    sc["sources"] = [sg.pencil_beam((0.3, 0.6, 1.0), (0, 0, -1), [490.0])]
    outs = batched(sc, 16, 40_000, max_events=1)
    tot = np.array([o["film"].sum() for o in outs])
    th = math.tan(math.radians(22.5))
    A = (2 * th) ** 2 / (W * W)
    m, se = batch_mean_se(tot * A)
    st = 2.0
    s = (np.arange(20000) + 0.5) / 20000
    val = 0.0
    for si in s:
        x = np.array([0.3, 0.6, 1.0 - si])
        v = x - eye
        r = np.linalg.norm(v)
        cos_t = v[1] / r
        d = -v / r
        # distance to leave the unit cube toward the eye (through the -y face)
        texit = x[1] / -d[1]
        val += st * math.exp(-st * si) * math.exp(-st * texit) / (4 * math.pi * r * r * cos_t ** 3)
    val /= 20000
    assert abs(m - val) <= 3 * se, (m, val, se)


def test_lambertian_wall_and_light_connections_are_exact():
    """Deterministic checks of the Lambertian vertex intensity rho cos/pi: a pencil beam hitting a
    diffuse floor seen by an ortho camera from above, and a point Lambertian light seen by a
    pinhole."""
    W = 8
    sensor = sg.ortho_sensor(W, W, (0, 0, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1))
    dyes = sg.make_dyes([490.0], [15.0], [620.0], [15.0], eps=[0.0], qy=[0.0])
    sc = slab_scene(1000, dyes=dyes, sensor=sensor)
    sc["medium"]["wall_mask"] = 1 << sg.FACE_NZ
    sc["medium"]["wall_albedo"] = 0.7
    sc["sources"] = [sg.pencil_beam((0.56, 0.56, 1.0), (0, 0, -1), [490.0])]
    r = oracle.render(sc, max_events=1)
    px = int(0.56 * W)
    rho = float(0.7)
    assert abs(r["film"][px, px, bin_of(490)] - rho / math.pi * W * W) < 1e-9
    # after the bounce, the photon escapes: top-face share is the form factor of the top square
    # from the floor centre-ish point (corner formula, four quadrants)

    def f_corner(X, Y):
        return (X / math.sqrt(1 + X * X) * math.atan(Y / math.sqrt(1 + X * X))
                + Y / math.sqrt(1 + Y * Y) * math.atan(X / math.sqrt(1 + Y * Y))) / (2 * math.pi)
    F = (f_corner(0.56, 0.56) + f_corner(0.44, 0.56) + f_corner(0.56, 0.44)
         + f_corner(0.44, 0.44))
    n = 200_000
    r = oracle.render(sc, n_paths=n, max_events=1)
    top = r["face"][0, sg.FACE_PZ].sum()
    assert abs(top - rho * F) <= 3 * rho * binomial_se(F, n), (top, rho * F)
    assert abs(r["face"].sum() - rho) < 1e-12
    # point Lambertian light on the floor facing +z, pinhole camera above
    eye = np.array([0.5, 0.5, 3.0])
    cam = sg.pinhole_sensor(W, W, eye, (1, 0, 0), (0, 1, 0), (0, 0, -1), 30.0)
    sc2 = slab_scene(100, dyes=dyes, sensor=cam)
    p = np.array([0.6, 0.45, 0.0])
    sc2["sources"] = [sg.rect_source("lambertian", p, (0, 0, 0), (0, 0, 0), (0, 0, 1), [490.0])]
    r = oracle.render(sc2, max_events=0)
    v = p - eye
    rr = np.linalg.norm(v)
    cos_t = -v[2] / rr
    th = math.tan(math.radians(15.0))
    A = (2 * th) ** 2 / (W * W)
    expect = (cos_t / math.pi) / (A * rr * rr * cos_t ** 3)
    assert abs(r["film"].sum() - expect) < 1e-9 * expect


def test_analog_and_weighted_modes_agree():
    """Both ways of applying QY (and the roulette that follows) estimate the same tallies."""
    sc = sg.cfg1_homogeneous_cube()
    a = batched(sc, 16, 6000, analog=1)
    w = batched(sc, 16, 6000, analog=0)
    for key in ("face", "emitted"):
        ma, sa = batch_mean_se([o[key].sum(axis=-1) for o in a])
        mw, sw = batch_mean_se([o[key].sum(axis=-1) for o in w])
        z = (ma - mw) / np.sqrt(sa ** 2 + sw ** 2 + 1e-300)
        assert np.abs(z[np.isfinite(z)]).max() < 4.0, (key, z)


def test_concentration_raises_fluorescence():
    """Sec. 5 (vials at 0.1/1/10 g/L): more dye gives more escaping fluorescence while the cube
    stays optically thin at the excitation line."""
    vals = []
    for c in (0.01, 0.1, 1.0):
        sc = sg.cfg1_homogeneous_cube(n_paths=40_000)
        sc["medium"]["conc_uniform"] = np.array([c], np.float32)
        vals.append(oracle.render(sc)["face"][1].sum())
    assert vals[0] < vals[1] < vals[2]


def test_thread_count_does_not_change_results():
    sc = sg.cfg1_homogeneous_cube(n_paths=5000)
    a = oracle.render(sc, n_threads=1, path_events=True)
    b = oracle.render(sc, n_threads=4, path_events=True)
    assert (a["path_events"] == b["path_events"]).all()
    assert np.allclose(a["face"], b["face"], rtol=1e-12, atol=1e-15)
    assert np.allclose(a["film"], b["film"], rtol=1e-10, atol=1e-12)
    assert a["counters"] == b["counters"]


# ------------------------------------------------------------------------------------------
# Local (macro-cell) majorants: the same estimator with fewer null collisions


def test_macro_cell_flight_reproduces_uncollided_transmission():
    """Delta tracking against per-cell majorants still samples the exact free-flight law (Eq. 6):
    the uncollided transmission through a random grid with a solvent mask matches
    exp(-column sum) for several cell sizes, with no majorant violation."""
    rng = np.random.default_rng(15)
    n = 12
    conc = rng.uniform(0.0, 2.0, size=(2, n, n, n)).astype(np.float32)
    conc[:, :, :, : n // 2] *= 0.05
    solvent = (rng.random((n, n, n)) < 0.6).astype(np.uint8)
    dyes = sg.make_dyes([490.0, 500.0], [15.0, 30.0], [620.0, 650.0], [15.0, 15.0],
                        eps=[0.3, 0.25], qy=[0.5, 0.5])
    x, y = 0.31, 0.64
    sc = {"spectrum": sg.spectrum(), "dyes": dyes,
          "medium": sg.grid_medium(conc, solvent, sigma_s=0.6),
          "sources": [sg.pencil_beam((x, y, 1.0), (0, 0, -1), [490.0])],
          "sensor": sg.no_sensor(), "params": sg.params(200_000, seed=4)}
    b = bin_of(490)
    exact = math.exp(-oracle.optical_depth(sc, np.array([x, y, 1.0]), np.array([0, 0, -1.0]), 1.0,
                                           b))
    for cell in (1, 3, 5, 12):
        r = oracle.render(sc, max_events=0, macro_cell=cell)
        T = r["face"][:, sg.FACE_NZ, :].sum()
        assert abs(T - exact) <= 3 * binomial_se(exact, 200_000), (cell, T, exact)
        assert r["counters"]["majorant_violations"] == 0


def test_macro_cell_render_matches_global_majorant_render():
    """Cornell box: local and global majorants estimate the same tallies and film (independent
    paths, batch-means z), with far fewer tracking steps."""
    sc = sg.cfg2_cornell_box(width=16, height=16, grid=32, n_paths=1)
    K, n = 16, 3000
    a = batched(sc, K, n)
    b = [oracle.render(sc, n_paths=n, path_offset=k * n, seed=11, macro_cell=4) for k in range(K)]
    for key in ("face", "emitted"):
        ma, sa = batch_mean_se([o[key].sum() for o in a])
        mb, sb = batch_mean_se([o[key].sum() for o in b])
        assert abs(ma - mb) <= 3 * math.sqrt(sa ** 2 + sb ** 2), (key, ma, mb)
    ma, sa = batch_mean_se([o["film"].sum() for o in a])
    mb, sb = batch_mean_se([o["film"].sum() for o in b])
    assert abs(ma - mb) <= 3 * math.sqrt(sa ** 2 + sb ** 2)
    steps_a = sum(o["counters"]["steps"] for o in a)
    steps_b = sum(o["counters"]["steps"] for o in b)
    assert steps_b < 0.5 * steps_a
    assert all(o["counters"]["majorant_violations"] == 0 for o in b)


# ------------------------------------------------------------------------------------------
# Empty-space leaps after null collisions (memoryless free flights)


def test_empty_space_leaps_reproduce_uncollided_transmission():
    """A beam crossing a grid whose matter fills only some regions (solvent mask and dyes zero
    elsewhere): leaving empty cubes after nulls keeps the exact uncollided transmission."""
    rng = np.random.default_rng(21)
    n = 16
    conc = rng.uniform(0.0, 2.0, size=(1, n, n, n)).astype(np.float32)
    solvent = np.zeros((n, n, n), np.uint8)
    solvent[4:7, :, :] = 1
    solvent[11:13, :, :] = 1
    conc[0][solvent == 0] = 0.0
    dyes = sg.make_dyes([490.0], [15.0], [620.0], [15.0], eps=[0.5], qy=[0.5])
    x, y = 0.43, 0.58
    sc = {"spectrum": sg.spectrum(), "dyes": dyes,
          "medium": sg.grid_medium(conc, solvent, sigma_s=1.5),
          "sources": [sg.pencil_beam((x, y, 1.0), (0, 0, -1), [490.0])],
          "sensor": sg.no_sensor(), "params": sg.params(200_000, seed=6)}
    exact = math.exp(-oracle.optical_depth(sc, np.array([x, y, 1.0]), np.array([0, 0, -1.0]), 1.0,
                                           bin_of(490)))
    base = oracle.render(sc, max_events=0)
    for cell in (1, 2, 4):
        r = oracle.render(sc, max_events=0, skip_cell=cell)
        T = r["face"][:, sg.FACE_NZ, :].sum()
        assert abs(T - exact) <= 3 * binomial_se(exact, 200_000), (cell, T, exact)
        if cell == 1:  # larger cells (with their halo) all touch the matter slabs here
            assert r["counters"]["steps"] < base["counters"]["steps"]


def test_empty_space_leaps_match_plain_tracking_on_cornell_box():
    sc = sg.cfg2_cornell_box(width=16, height=16, grid=32, n_paths=1)
    K, n = 16, 3000
    a = batched(sc, K, n)
    b = [oracle.render(sc, n_paths=n, path_offset=k * n, seed=13, skip_cell=2) for k in range(K)]
    for key in ("face", "emitted", "film"):
        ma, sa = batch_mean_se([o[key].sum() for o in a])
        mb, sb = batch_mean_se([o[key].sum() for o in b])
        assert abs(ma - mb) <= 3 * math.sqrt(sa ** 2 + sb ** 2), (key, ma, mb)
    assert sum(o["counters"]["steps"] for o in b) < 0.6 * sum(o["counters"]["steps"] for o in a)
