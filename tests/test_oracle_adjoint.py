"""Pins of the oracle's reference gradient (CPU, no GPU).

The gradient is that of L = sum_j adj_j I_j for the frozen-sampling estimator I (decisions sampled
at theta_0, tallies weighted by the likelihood ratio p_theta / p_theta_0), so central finite
differences with common random numbers are smooth per path and must agree to O(h^2). The frozen
estimator itself is pinned to the plainly resampled one, and the transmittance derivative to the
closed form d/dc exp(-sigma_a c h) = -sigma_a h exp(-sigma_a c h).
"""
import math

import numpy as np

import oracle
import scenegen as sg
from tests.stats import batch_mean_se


def small_adjoint_scene(n=8, W=8, seed=0, sigma_s=10.0):
    rng = np.random.default_rng(100 + seed)
    conc = np.stack([sg.blob_field(rng, n, 6, (1.0, 2.5)) for _ in range(2)])
    conc /= conc.reshape(2, -1).mean(axis=1)[:, None, None, None]
    dyes = sg.make_dyes([470.0, 560.0], [15.0, 15.0], [520.0, 610.0], [20.0, 20.0],
                        eps=[1.5, 1.0], qy=[0.8, 0.6])
    return {"spectrum": sg.spectrum(), "dyes": dyes,
            "medium": sg.grid_medium(conc.astype(np.float32), None, sigma_s=sigma_s),
            "sources": [sg.rect_source("collimated", (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1),
                                       [470.0, 560.0])],
            "sensor": sg.ortho_sensor(W, W, (0, 0, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1)),
            "params": sg.params(3000, seed=1)}


def loss(r, adj):
    return float((r["film"] * adj).sum())


def test_frozen_render_without_perturbation_is_the_plain_render():
    sc = small_adjoint_scene()
    a = oracle.render(sc, majorant_scale=1.25, n_threads=1)
    b = oracle.render(sc, majorant_scale=1.25, frozen=True, pert=(0, 5, 0.0, 0.0), n_threads=1)
    assert np.array_equal(a["film"], b["film"])
    assert np.array_equal(a["face"], b["face"])


def test_frozen_estimator_matches_resampled_perturbed_scene():
    """Both estimate the perturbed scene without bias. The frozen weights are products of
    per-decision ratios, so their variance grows quickly with the perturbation: a 5 % change of
    sigma_s keeps it small enough to pin the mean."""
    sc = small_adjoint_scene()
    K, n = 16, 4000
    pert = (None, 0, 0.0, 0.5)  # sigma_s 10 -> 10.5
    fz = [oracle.render(sc, n_paths=n, path_offset=k * n, majorant_scale=1.5, frozen=True,
                        pert=pert) for k in range(K)]
    rs = [oracle.render(sc, n_paths=n, path_offset=k * n, seed=77, majorant_scale=1.5,
                        pert=pert) for k in range(K)]
    for key in ("face", "film"):
        mf, sf = batch_mean_se([o[key].sum() for o in fz])
        mr, sr = batch_mean_se([o[key].sum() for o in rs])
        assert abs(mf - mr) <= 3 * math.sqrt(sf ** 2 + sr ** 2), (key, mf, mr)


def test_adjoint_matches_frozen_central_differences():
    sc = small_adjoint_scene()
    rng = np.random.default_rng(3)
    adj = rng.normal(size=(8, 8, sg.N_BINS))
    ms = 1.25
    gc, gs = oracle.adjoint(sc, adj, majorant_scale=ms)
    conc = sc["medium"]["conc"]
    D, nz, ny, nx = conc.shape
    scale = np.abs(gc).max()
    checked = 0
    for _ in range(12):
        d = int(rng.integers(0, D))
        v = int(rng.integers(0, nz * ny * nx))
        c0 = float(conc[d].reshape(-1)[v])
        h = 1e-3 * max(c0, 1e-2)
        lp = loss(oracle.render(sc, majorant_scale=ms, frozen=True, pert=(d, v, +h, 0.0)), adj)
        lm = loss(oracle.render(sc, majorant_scale=ms, frozen=True, pert=(d, v, -h, 0.0)), adj)
        fd = (lp - lm) / (2 * h)
        g = gc[d].reshape(-1)[v]
        assert abs(fd - g) <= 1e-4 * abs(g) + 1e-7 * scale, (d, v, fd, g)
        checked += g != 0.0
    assert checked >= 6
    # sigma_s enters every scatter of a path: a path with k of them carries (1 + h/sigma_s)^k, so
    # the central difference errs by about k^2 (h/sigma_s)^2 / 6; it must shrink as O(h^2)
    for rel, tol in ((1e-3, 1e-3), (1e-5, 1e-6)):
        hs = rel * sc["medium"]["sigma_s"]
        lp = loss(oracle.render(sc, majorant_scale=ms, frozen=True, pert=(None, 0, 0.0, +hs)), adj)
        lm = loss(oracle.render(sc, majorant_scale=ms, frozen=True, pert=(None, 0, 0.0, -hs)), adj)
        fd = (lp - lm) / (2 * hs)
        assert abs(fd - gs) <= tol * abs(gs) + 1e-12, (rel, fd, gs)


def test_transmittance_gradient_closed_form_column():
    """Point Lambertian light on the floor of a non-scattering absorbing grid, ortho camera above:
    the film pixel holds I = exp(-sum_v sigma_a c_v h) / (pi A_pix) and dI/dc_v = -sigma_a h I on
    the voxels of the light's column, zero elsewhere."""
    n, W = 6, 6
    rng = np.random.default_rng(9)
    conc = rng.uniform(0.2, 1.5, size=(1, n, n, n)).astype(np.float32)
    dyes = sg.make_dyes([490.0], [15.0], [620.0], [15.0], eps=[0.7], qy=[0.0])
    p = (0.55, 0.25, 0.0)
    sc = {"spectrum": sg.spectrum(), "dyes": dyes, "medium": sg.grid_medium(conc, None),
          "sources": [sg.rect_source("lambertian", p, (0, 0, 0), (0, 0, 0), (0, 0, 1), [490.0])],
          "sensor": sg.ortho_sensor(W, W, (0, 0, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1)),
          "params": sg.params(200, seed=2)}
    b = int(math.ceil((490 - sg.LAMBDA0) / sg.DLAMBDA - 0.5))
    px, py = int(p[0] * W), int(p[1] * W)
    ix, iy = int(p[0] * n), int(p[1] * n)
    sa = float(dyes["eps"][0]) * float(dyes["abs_shape"][0, b])
    tau = sa * conc[0, :, iy, ix].astype(np.float64).sum() / n
    I = math.exp(-tau) / math.pi * W * W
    r = oracle.render(sc)
    assert abs(r["film"][py, px, b] - I) < 1e-9 * I
    adj = np.zeros((W, W, sg.N_BINS))
    adj[py, px, b] = 1.0
    gc, gs = oracle.adjoint(sc, adj)
    want = np.zeros_like(gc)
    want[0, :, iy, ix] = -sa / n * I
    assert np.allclose(gc, want, rtol=1e-9, atol=1e-12 * I)
    # sigma_t contains sigma_s (zero here) everywhere, so dI/dsigma_s = -(column length) I
    assert abs(gs + 1.0 * I) < 1e-9 * I
