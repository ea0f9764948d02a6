"""Pins of the oracle's refractive interfaces and glossy walls (CPU, no GPU).

The paper renders dye solutions in glass vials and a glossy Cornell box (Sec. 5) without saying
how it models either; the oracle takes the physically standard choices: smooth dielectric faces
(Fresnel reflection of unpolarised light, Snell refraction, total internal reflection) and a wall
BRDF of a diffuse lobe plus a normalised Phong lobe about the mirror direction. Each pin is a
closed form or a quadrature reached by a different route than the oracle's code:
  - the slab series of a beam at normal incidence bouncing between two faces (F0 of the textbook
    normal-incidence formula, Beer-Lambert between bounces, Eq. 6);
  - an oblique beam through a wide slab, with the reflectances from the angle form of Fresnel's
    equations (sin^2 / tan^2 of the sum and difference angles) and Stokes' reciprocity;
  - the fraction of isotropically re-emitted photons trapped for ever by total internal reflection
    in a cube (a direction is trapped iff every |component| is below the critical cosine);
  - the glossy lobe's energy and the share leaving through the top face, by quadrature;
  - the film of a glossy floor seen head-on by an orthographic camera, exact per photon.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
import scenegen as sg
from tests.stats import binomial_se


def _box_scene(dyes, medium, sources, sensor=None, n_paths=100_000, **kw):
    return {"spectrum": sg.spectrum(), "dyes": dyes, "medium": medium, "sources": sources,
            "sensor": sensor or sg.no_sensor(), "params": sg.params(n_paths, **kw)}


def _clear_dye():
    return sg.make_dyes([490.0], [15.0], [650.0], [15.0], eps=[0.0], qy=[0.0])


def fresnel_angles(theta_i, n1, n2):
    """Unpolarised reflectance from the angle form of Fresnel's equations."""
    st = n1 / n2 * math.sin(theta_i)
    if st >= 1.0:
        return 1.0
    tt = math.asin(st)
    if theta_i == 0.0:
        return ((n1 - n2) / (n1 + n2)) ** 2
    rs = math.sin(theta_i - tt) ** 2 / math.sin(theta_i + tt) ** 2
    rp = math.tan(theta_i - tt) ** 2 / math.tan(theta_i + tt) ** 2
    return 0.5 * (rs + rp)


def test_normal_incidence_slab_series_with_absorption():
    """Pencil beam into a non-scattering absorbing cube of index 1.5: it bounces between the two
    faces, losing 1 - F0 at each and e^-tau between them:
    T = (1-F0)^2 e^-tau / (1 - F0^2 e^-2tau), R = F0 + (1-F0)^2 F0 e^-2tau / (1 - F0^2 e^-2tau)."""
    n, tau, N = 1.5, 1.0, 200_000
    med = sg.homogeneous_medium(1, conc=1.0, sigma_a0=tau)
    med["ior"] = n
    sc = _box_scene(_clear_dye(), med, [sg.pencil_beam((0.5, 0.5, 1.0), (0, 0, -1), [490.0])],
                    n_paths=N)
    r = oracle.render(sc, film=False)
    F0 = ((n - 1) / (n + 1)) ** 2
    e1, e2 = math.exp(-tau), math.exp(-2 * tau)
    T = (1 - F0) ** 2 * e1 / (1 - F0 ** 2 * e2)
    R = F0 + (1 - F0) ** 2 * F0 * e2 / (1 - F0 ** 2 * e2)
    got_T = r["face"][0, sg.FACE_NZ].sum()
    got_R = r["face"][0, sg.FACE_PZ].sum()
    assert abs(got_T - T) <= 4 * binomial_se(T, N), (got_T, T)
    assert abs(got_R - R) <= 4 * binomial_se(R, N), (got_R, R)
    assert abs(r["absorbed"][1].sum() - (1 - T - R)) <= 4 * binomial_se(1 - T - R, N)
    assert r["face"][:, :4].sum() == 0.0 and r["face"][1].sum() == 0.0
    assert r["counters"]["iface_reflections"] > 0


def test_oblique_beam_through_a_wide_slab():
    """A beam at 60 deg into the top of a 10 x 10 x 1 cm slab of index 1.5 absorbing sigma_a. Inside
    it runs at theta_t = asin(sin 60 / 1.5), so each pass is 1 / cos theta_t long (tau per pass),
    and meets the bottom and the top at theta_t, where the reflectance equals the entry one R
    (Stokes): the slab series gives the bottom (1-R)^2 e^-tau / (1 - R^2 e^-2tau) and the top
    R + (1-R)^2 R e^-2tau / (1 - R^2 e^-2tau). The side faces are reached only after seven passes
    (R^7 ~ 5e-8). Without absorption the two shares are (1 - R)/(1 + R) and 2R/(1 + R)."""
    n, N = 1.5, 200_000
    th = math.radians(60.0)
    R = fresnel_angles(th, 1.0, n)
    tt = math.asin(math.sin(th) / n)
    assert abs(fresnel_angles(tt, n, 1.0) - R) < 1e-12
    for sa in (0.0, 0.3):
        med = sg.homogeneous_medium(1, conc=1.0, sigma_a0=sa, hi=(10.0, 10.0, 1.0))
        med["ior"] = n
        d = (math.sin(th), 0.0, -math.cos(th))
        sc = _box_scene(_clear_dye(), med, [sg.pencil_beam((5.0, 5.0, 1.0), d, [490.0])],
                        n_paths=N)
        r = oracle.render(sc, film=False)
        e1 = math.exp(-sa / math.cos(tt))
        e2 = e1 * e1
        bottom = (1 - R) ** 2 * e1 / (1 - R * R * e2)
        top = R + (1 - R) ** 2 * R * e2 / (1 - R * R * e2)
        got_b, got_t = r["face"][0, sg.FACE_NZ].sum(), r["face"][0, sg.FACE_PZ].sum()
        assert abs(got_b - bottom) <= 4 * binomial_se(bottom, N), (sa, got_b, bottom)
        assert abs(got_t - top) <= 4 * binomial_se(top, N), (sa, got_t, top)
        if sa == 0.0:
            assert abs(bottom - (1 - R) / (1 + R)) < 1e-12 and abs(r["face"].sum() - 1.0) < 1e-9


def test_refracted_beam_drifts_by_tan_theta_t():
    """The same beam 0.5 cm from the -x edge of a 2 cm wide, strongly absorbing slab: refracted at
    theta_t it drifts tan(theta_t) = 0.707 cm per pass, so it leaves through the bottom at x = 1.21
    and, once reflected there, through the top at x = 1.91; only after a second internal
    reflection (weight R^2 e^-2tau ~ 1e-5) could it reach the +x face. A wrong refraction angle
    sends it into the side face on the first pass."""
    n, N, sa = 1.5, 200_000, 3.0
    th = math.radians(60.0)
    R = fresnel_angles(th, 1.0, n)
    tt = math.asin(math.sin(th) / n)
    assert abs(math.tan(tt) - math.sqrt(0.5)) < 1e-12
    med = sg.homogeneous_medium(1, conc=1.0, sigma_a0=sa, hi=(2.0, 10.0, 1.0))
    med["ior"] = n
    d = (math.sin(th), 0.0, -math.cos(th))
    sc = _box_scene(_clear_dye(), med, [sg.pencil_beam((0.5, 5.0, 1.0), d, [490.0])], n_paths=N)
    r = oracle.render(sc, film=False)
    e1 = math.exp(-sa / math.cos(tt))
    bottom = (1 - R) ** 2 * e1
    top = R + (1 - R) ** 2 * R * e1 * e1
    got_b, got_t = r["face"][0, sg.FACE_NZ].sum(), r["face"][0, sg.FACE_PZ].sum()
    assert abs(got_b - bottom) <= 4 * binomial_se(bottom, N) + 1e-5, (got_b, bottom)
    assert abs(got_t - top) <= 4 * binomial_se(top, N) + 1e-5, (got_t, top)
    assert r["face"][0, sg.FACE_PX].sum() <= 4 * binomial_se(1e-5, N) + 1e-5


def trapped_fraction(n):
    """P(|w_x|, |w_y|, |w_z| < c) for w uniform on the sphere, c = sqrt(1 - 1/n^2): integrate over
    mu = w_z the azimuth measure where both in-plane components stay below c."""
    c = math.sqrt(1.0 - 1.0 / n ** 2)

    def arc(mu):
        s = math.sqrt(max(0.0, 1.0 - mu * mu))
        if s <= c:
            return 2.0 * math.pi
        a = math.acos(c / s)   # |cos phi| < c / s  <=>  phi in (a, pi - a) (mod pi)
        b = math.asin(c / s)   # |sin phi| < c / s  <=>  phi in (-b, b) (mod pi)
        return 4.0 * max(0.0, b - a)

    val, _ = integrate.quad(arc, -c, c, limit=200, points=[-math.sqrt(1 - c * c), math.sqrt(1 - c * c)])
    return val / (4.0 * math.pi)


def test_total_internal_reflection_traps_the_predicted_fraction():
    """A thin dye in a non-scattering cube of index 1.5 absorbs the normal beam (after the slab
    series at 490 nm) and re-emits at 650 nm, where nothing absorbs. Specular reflections on a box
    only flip signs, so an emitted direction whose three |components| are all below the critical
    cosine is trapped for ever (it ends at the event cap); every other one escapes."""
    n, tau, N = 1.5, 0.5, 100_000
    dyes = sg.make_dyes([490.0], [15.0], [650.0], [15.0], eps=[tau], qy=[1.0])
    med = sg.homogeneous_medium(1, conc=1.0)
    med["ior"] = n
    sc = _box_scene(dyes, med, [sg.pencil_beam((0.5, 0.5, 1.0), (0, 0, -1), [490.0])],
                    n_paths=N, max_events=20_000)
    r = oracle.render(sc, film=False)
    F0 = ((n - 1) / (n + 1)) ** 2
    e1, e2 = math.exp(-tau), math.exp(-2 * tau)
    A = (1 - F0) * (1 - e1) * (1 + F0 * e1) / (1 - F0 ** 2 * e2)
    P = trapped_fraction(n)
    assert 0.05 < P < 0.5
    got_abs = r["absorbed"][0].sum()
    assert abs(got_abs - A) <= 4 * binomial_se(A, N), (got_abs, A)
    cap = r["counters"]["cap_hits"] / N
    assert abs(cap - A * P) <= 4 * binomial_se(A * P, N), (cap, A * P)
    fl = r["face"][1].sum()
    assert abs(fl - A * (1 - P)) <= 4 * binomial_se(A * (1 - P), N), (fl, A * (1 - P))
    # the escaped fluorescence is the emission line, at 650 nm
    assert r["face"][1].sum(axis=0).argmax() == int(math.ceil((650 - sg.LAMBDA0) / sg.DLAMBDA - 0.5))


def test_trapped_fraction_quadrature_against_brute_force_directions():
    rng = np.random.default_rng(0)
    w = rng.normal(size=(2_000_000, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    for n in (1.33, 1.5, 2.0):
        c = math.sqrt(1 - 1 / n ** 2)
        mc = float((np.abs(w) < c).all(axis=1).mean())
        assert abs(mc - trapped_fraction(n)) < 1e-3, (n, mc, trapped_fraction(n))


def _glossy_floor_scene(theta_deg, rho, g, e, N, phi_deg=0.0):
    th, ph = math.radians(theta_deg), math.radians(phi_deg)
    med = sg.homogeneous_medium(1, conc=0.0, wall_mask=1 << sg.FACE_NZ, wall_albedo=rho)
    med["wall_gloss"] = g
    med["wall_exponent"] = e
    d = (math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), -math.cos(th))
    # a beam starting inside the empty box, 0.25 cm above the floor, aimed at the floor centre
    z0 = 0.25
    o = (0.5 - z0 * math.tan(th) * math.cos(ph), 0.5 - z0 * math.tan(th) * math.sin(ph), z0)
    assert all(0.0 <= v <= 1.0 for v in o)
    cam = sg.ortho_sensor(8, 8, (0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0))
    return _box_scene(_clear_dye(), med, [sg.pencil_beam(o, d, [490.0])], cam, n_paths=N)


def _lobe_integral(theta, e, region=None, phi=0.0):
    """Quadrature of (e + 2)/(2 pi) cos^e alpha cos theta_o over the outgoing directions above the
    floor (optionally only those in `region`), in a frame of its own about the mirror direction
    r = (sin theta cos phi, sin theta sin phi, cos theta)."""
    r = np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)])
    t1 = np.array([math.cos(theta) * math.cos(phi), math.cos(theta) * math.sin(phi), -math.sin(theta)])
    t2 = np.cross(r, t1)
    na, nph = 1200, 1200
    a = (np.arange(na) + 0.5) * (math.pi / 2) / na
    ph = (np.arange(nph) + 0.5) * 2 * math.pi / nph
    A, PH = np.meshgrid(a, ph, indexing="ij")
    w = (np.sin(A) * np.cos(PH))[..., None] * t1 + (np.sin(A) * np.sin(PH))[..., None] * t2 + \
        np.cos(A)[..., None] * r
    co = w[..., 2]
    f = (e + 2) / (2 * math.pi) * np.cos(A) ** e * np.clip(co, 0.0, None) * np.sin(A)
    if region is not None:
        f = f * region(w)
    return float(f.sum() * (math.pi / 2 / na) * (2 * math.pi / nph))


@pytest.mark.parametrize("theta_deg,phi_deg,e", [(0.0, 0.0, 20.0), (30.0, 0.0, 20.0),
                                                 (60.0, 0.0, 20.0), (40.0, 35.0, 20.0),
                                                 (50.0, -60.0, 2.0), (0.0, 0.0, 2.0)])
def test_glossy_lobe_energy_and_top_face_share(theta_deg, phi_deg, e):
    """One glossy bounce on the floor of an otherwise open box (weighted mode): the escaped weight
    is the directional albedo rho [(1 - g) + g a(theta)], a(theta) the lobe integral above the
    floor; the share leaving through the top face (|w_x|, |w_y| < w_z / 2 from the floor centre)
    follows the same quadrature restricted to that cone. Incidence out of the xz plane checks the
    lobe's frame, a low exponent its sampling density."""
    rho, g, N = 0.8, 0.6, 200_000
    th, ph = math.radians(theta_deg), math.radians(phi_deg)
    sc = _glossy_floor_scene(theta_deg, rho, g, e, N, phi_deg)
    r = oracle.render(sc, film=False)
    a = _lobe_integral(th, e, phi=ph)
    if theta_deg == 0.0:
        assert abs(a - 1.0) < 1e-4   # at normal incidence the lobe holds all its energy
    want = rho * ((1 - g) + g * a)
    got = r["face"][0].sum()
    # weights rho (diffuse) or rho (e+2)/(e+1) cos (glossy): SE from the two-point spread
    se = rho * (e + 2) / (e + 1) / math.sqrt(N)
    assert abs(got - want) <= 4 * se, (got, want)
    top = lambda w: ((np.abs(w[..., 0]) < 0.5 * w[..., 2]) & (np.abs(w[..., 1]) < 0.5 * w[..., 2]))
    a_top = _lobe_integral(th, e, top, phi=ph)
    # the diffuse share through the square: the solid-angle-weighted cosine integral
    d_top = _diffuse_square_fraction(0.5, 1.0)
    want_top = rho * ((1 - g) * d_top + g * a_top)
    got_top = r["face"][0, sg.FACE_PZ].sum()
    assert abs(got_top - want_top) <= 4 * se, (got_top, want_top)
    # and the side faces by symmetry-free bookkeeping: +x against -x for a beam heading +x
    if phi_deg == 0.0 and theta_deg > 0.0:
        px = lambda w: (w[..., 0] > 0.5 * w[..., 2]) & (np.abs(w[..., 1]) < w[..., 0])
        a_px = _lobe_integral(th, e, px, phi=ph)
        # the diffuse lobe sends the same share through each side face
        d_side = (1.0 - d_top) / 4
        want_px = rho * ((1 - g) * d_side + g * a_px)
        got_px = r["face"][0, sg.FACE_PX].sum()
        assert abs(got_px - want_px) <= 4 * se, (got_px, want_px)


def _diffuse_square_fraction(half, h):
    """Share of a cosine-weighted hemisphere leaving through a centred square of half-side `half`
    at height h: (1/pi) times the integral of cos(theta) over its solid angle."""
    def f(y, x):
        r2 = x * x + y * y + h * h
        return h * h / (math.pi * r2 * r2)
    val, _ = integrate.dblquad(f, -half, half, -half, half)
    return val


def test_glossy_floor_film_seen_head_on():
    """Every photon hits the floor centre; the orthographic camera above records
    rho [(1 - g)/pi + g (e + 2)/(2 pi) cos^e theta] / A_pix in the centre pixel and nothing else."""
    rho, g, e = 0.8, 0.6, 20.0
    for theta_deg in (0.0, 25.0):
        sc = _glossy_floor_scene(theta_deg, rho, g, e, 2000)
        r = oracle.render(sc)
        th = math.radians(theta_deg)
        want = rho * ((1 - g) / math.pi + g * (e + 2) / (2 * math.pi) * math.cos(th) ** e) * 64
        film = r["film"]
        assert film[4, 4].sum() == pytest.approx(want, rel=1e-9)
        film[4, 4] = 0.0
        assert film.sum() == 0.0


def test_film_through_a_dielectric_face_at_normal_incidence():
    """A cuvette of index n with a Lambertian floor, seen head-on through its top face: the beam
    enters (1 - F0 of it), lights the floor centre, and the floor's first-bounce radiance reaches
    the camera through the top face with the transmitted fraction 1 - F0 and the 1/n^2 of radiance
    leaving a denser medium. With the event cap at 1 nothing else reaches the film, so the centre
    pixel holds (1 - F0)^2 rho / (pi n^2) / A_pix (binomial in the entry coin)."""
    rho, N = 0.7, 100_000
    for n in (1.33, 1.5):
        med = sg.homogeneous_medium(1, conc=0.0, wall_mask=1 << sg.FACE_NZ, wall_albedo=rho)
        med["ior"] = n
        cam = sg.ortho_sensor(8, 8, (0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0),
                              (0.0, 0.0, 1.0))
        sc = _box_scene(_clear_dye(), med, [sg.pencil_beam((0.5, 0.5, 1.0), (0, 0, -1), [490.0])],
                        cam, n_paths=N, max_events=1)
        r = oracle.render(sc)
        F0 = ((n - 1) / (n + 1)) ** 2
        unit = rho / (math.pi * n * n) * 64
        want = (1 - F0) ** 2 * unit
        got = r["film"][4, 4].sum()
        assert abs(got - want) <= 4 * unit * binomial_se(1 - F0, N), (n, got, want)
        film = r["film"]
        film[4, 4] = 0.0
        assert film.sum() == 0.0


def test_interfaces_are_rejected_where_they_are_not_modelled():
    med = sg.homogeneous_medium(1, conc=1.0, sigma_s=1.0)
    med["ior"] = 1.5
    pin = sg.pinhole_sensor(8, 8, eye=(0.5, -2.0, 0.5), right=(1, 0, 0), up=(0, 0, 1),
                            forward=(0, 1, 0), fov_y_deg=30.0)
    sc = _box_scene(_clear_dye(), med, [sg.pencil_beam((0.5, 0.5, 1.0), (0, 0, -1), [490.0])],
                    pin, n_paths=10)
    with pytest.raises(ValueError):
        oracle.render(sc)
    sc["sensor"] = sg.ortho_sensor(8, 8, (0, 0, 0), (1, 0, 0), (0, 0, 1), (0.0, -0.6, 0.8))
    with pytest.raises(ValueError):
        oracle.render(sc)
    sc["sensor"] = sg.ortho_sensor(8, 8, (0, 0, 0), (1, 0, 0), (0, 0, 1), (0.0, -1.0, 0.0))
    oracle.render(sc)
    with pytest.raises(ValueError):
        oracle.render(sc, hero=2)
