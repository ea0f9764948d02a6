"""Path-replay adjoint on the GPU (flr_adjoint, FluoroRender) against the oracle's reference
gradient, a closed form, central differences with common random numbers, and its own linearity.

The oracle's gradient (tests/test_oracle_adjoint.py) is pinned to frozen-sampling central
differences and a closed form; the GPU's must agree with it statistically (the GPU estimates each
transmittance by ratio tracking, the oracle evaluates it exactly, so per path they differ).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from paper_1706_03024_gb300 import native as N
from paper_1706_03024_gb300.scene import FluoroRender, Scene
from tests.gpu_common import require_gpu
from tests.stats import batch_mean_se, parity_verdict

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def adjoint_scene(n=12, W=12, sigma_s=10.0, n_paths=4000):
    rng = np.random.default_rng(100)
    conc = np.stack([sg.blob_field(rng, n, 8, (1.5, 3.5)) for _ in range(2)])
    conc /= conc.reshape(2, -1).mean(axis=1)[:, None, None, None]
    dyes = sg.make_dyes([470.0, 560.0], [15.0, 15.0], [520.0, 610.0], [20.0, 20.0],
                        eps=[1.5, 1.0], qy=[0.8, 0.6])
    return {"spectrum": sg.spectrum(), "dyes": dyes,
            "medium": sg.grid_medium(conc.astype(np.float32), None, sigma_s=sigma_s),
            "sources": [sg.rect_source("collimated", (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1),
                                       [470.0, 560.0])],
            "sensor": sg.ortho_sensor(W, W, (0, 0, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1)),
            "params": sg.params(n_paths, seed=1)}


def gpu_adjoint(S, adj, n, offset=0, seed=None, macro_cell=0, margin=0.0, form="wavefront_warp"):
    gc = torch.zeros(S.conc_t.shape, dtype=torch.float32, device="cuda")
    gs = torch.zeros(1, dtype=torch.float32, device="cuda")
    S.adjoint(torch.from_numpy(adj.astype(np.float32)).cuda(), gc, gs, n_paths=n,
              path_offset=offset, seed=seed, macro_cell=macro_cell, majorant_margin=margin,
              form=form)
    return gc.double().cpu().numpy(), float(gs.item())


@pytest.mark.parametrize("sigma_s,n,macro_cell", [(10.0, 40_000, 0), (60.0, 20_000, 0),
                                                  (10.0, (1 << 21) + 4096, 0), (10.0, 40_000, 3)])
def test_warp_adjoint_equals_plain_replay(sigma_s, n, macro_cell):
    """The two-pass warp-regrouped replay evaluates the same per-path terms as the one-thread
    replay (same decisions, same ratio-tracking points, same suffix sums), so the gradients agree
    up to the order of the fp32 atomics. sigma_s = 60 gives paths with more connections than the
    per-path store holds (their later contributions are recomputed in pass 2); 2^21 + 4096 paths
    take two path chunks."""
    sc = adjoint_scene(sigma_s=sigma_s)
    S = Scene(sc)
    if sigma_s > 30:
        ev = torch.zeros(n, dtype=torch.int32, device="cuda")
        S.render(n_paths=n, path_events=ev, majorant_margin=0.1)
        assert int(ev.max()) > 40
    rng = np.random.default_rng(11)
    adj = rng.normal(size=(12, 12, sg.N_BINS))
    gp, sp = gpu_adjoint(S, adj, n, macro_cell=macro_cell, margin=0.1, form="plain")
    gw, sw = gpu_adjoint(S, adj, n, macro_cell=macro_cell, margin=0.1, form="wavefront_warp")
    scale = np.abs(gp).max()
    assert scale > 0
    assert np.allclose(gw, gp, rtol=1e-3, atol=1e-4 * scale), np.abs(gw - gp).max() / scale
    assert abs(sw - sp) <= 1e-4 * max(abs(sp), 1e-30) + 1e-6 * scale, (sw, sp)


# The score estimator needs sigma_bar > sigma_t wherever sigma_t depends on the parameters (a null
# that has probability 0 at theta_0 is never sampled although its probability changes with theta),
# so gradients are taken with a 10 % majorant margin, on both sides.
@pytest.mark.parametrize("macro_cell,margin", [(0, 0.1), (3, 0.1)])
def test_adjoint_matches_oracle_reference_gradient(macro_cell, margin):
    sc = adjoint_scene()
    S = Scene(sc)
    rng = np.random.default_rng(5)
    adj = rng.normal(size=(12, 12, sg.N_BINS))
    K, n = 16, 4000
    g = [gpu_adjoint(S, adj, n, k * n, macro_cell=macro_cell, margin=margin) for k in range(K)]
    o = [oracle.adjoint(sc, adj, n_paths=n, path_offset=k * n, macro_cell=macro_cell,
                        majorant_scale=1.0 + margin) for k in range(K)]
    mg, sg_ = batch_mean_se([x[0] for x in g])
    mo, so = batch_mean_se([x[0] for x in o])
    # a dye collision scores suffix / c: at voxels with a tiny concentration these are rare events
    # of huge weight, decided on a sliver of u that fp32 and fp64 round differently, so the
    # per-voxel comparison covers c >= 0.05 (mean 1); the per-dye totals below cover every voxel
    keep = sc["medium"]["conc"] >= 0.05
    if macro_cell == 0:
        v = parity_verdict(np.where(keep, mg, 0.0), np.where(keep, sg_, 0.0),
                           np.where(keep, mo, 0.0), np.where(keep, so, 0.0), check_chi2=False)
    else:
        # local majorants only 10 % above sigma_t make null scores -1/(sigma_bar - sigma_t) large
        # and rare: compare per-dye z-slabs (sums over x, y) instead of single voxels
        gs_ = np.stack([np.where(keep, x[0], 0.0).sum(axis=(2, 3)) for x in g])
        os_ = np.stack([np.where(keep, x[0], 0.0).sum(axis=(2, 3)) for x in o])
        a, sa = batch_mean_se(gs_)
        b, sb = batch_mean_se(os_)
        v = parity_verdict(a, sa, b, sb, check_chi2=False)
    assert v["ok"], v
    # the per-dye total and the sigma_s derivative
    for d in range(2):
        a, sa = batch_mean_se([x[0][d].sum() for x in g])
        b, sb = batch_mean_se([x[0][d].sum() for x in o])
        assert abs(a - b) <= 3 * math.hypot(sa, sb), (d, a, b)
    a, sa = batch_mean_se([x[1] for x in g])
    b, sb = batch_mean_se([x[1] for x in o])
    assert abs(a - b) <= 3 * math.hypot(sa, sb), (a, b)
    assert np.abs(mo).max() > 0


def test_adjoint_closed_form_column():
    """Lambertian point light on the floor of a non-scattering absorbing grid, ortho camera above:
    E[dI/dc_v] = -sigma_a h I on the light's column, and exactly zero elsewhere."""
    n, W = 6, 6
    rng = np.random.default_rng(9)
    conc = rng.uniform(0.2, 1.5, size=(1, n, n, n)).astype(np.float32)
    dyes = sg.make_dyes([490.0], [15.0], [620.0], [15.0], eps=[0.7], qy=[0.0])
    p = (0.55, 0.25, 0.0)
    sc = {"spectrum": sg.spectrum(), "dyes": dyes, "medium": sg.grid_medium(conc, None),
          "sources": [sg.rect_source("lambertian", p, (0, 0, 0), (0, 0, 0), (0, 0, 1), [490.0])],
          "sensor": sg.ortho_sensor(W, W, (0, 0, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1)),
          "params": sg.params(20000, seed=2)}
    b = int(math.ceil((490 - sg.LAMBDA0) / sg.DLAMBDA - 0.5))
    px, py = int(p[0] * W), int(p[1] * W)
    ix, iy = int(p[0] * n), int(p[1] * n)
    sa = float(dyes["eps"][0]) * float(dyes["abs_shape"][0, b])
    I = math.exp(-sa * conc[0, :, iy, ix].astype(np.float64).sum() / n) / math.pi * W * W
    adj = np.zeros((W, W, sg.N_BINS))
    adj[py, px, b] = 1.0
    S = Scene(sc)
    K, N = 16, 20000
    runs = [gpu_adjoint(S, adj, N, k * N) for k in range(K)]
    m, se = batch_mean_se([r[0] for r in runs])
    want = np.zeros_like(m)
    want[0, :, iy, ix] = -sa / n * I
    mask = np.zeros(m.shape, bool)
    mask[0, :, iy, ix] = True
    assert (m[~mask] == 0).all()
    assert np.all(np.abs(m[mask] - want[mask]) <= 3.5 * se[mask] + 1e-6 * I), (m[mask], want[mask])
    ms, ss = batch_mean_se([r[1] for r in runs])
    assert abs(ms + I) <= 3.5 * ss + 1e-6 * I


def test_autograd_function_matches_flr_adjoint():
    sc = adjoint_scene(n_paths=200_000)
    S = Scene(sc)
    conc = torch.from_numpy(sc["medium"]["conc"]).cuda()
    target = Scene(adjoint_scene(n_paths=200_000)).render(form="wavefront", seed=99).clone() * 1.3
    opts = {"n_paths": 200_000, "seed": 3}
    c = conc.clone().requires_grad_(True)
    s = torch.tensor(10.0, dtype=torch.float64, requires_grad=True)
    film = FluoroRender.apply(c, s, S, opts)
    loss = ((film.double() - target.double()) ** 2).sum()
    loss.backward()
    # backward equals flr_adjoint with adj = dL/dI = 2 (I - T)
    adj = (2.0 * (film.detach().double() - target.double())).float()
    gc = torch.zeros_like(conc)
    gs = torch.zeros(1, device="cuda")
    S.set_medium_values(conc, 10.0)
    S.adjoint(adj, gc, gs, majorant_margin=0.1, **opts)  # FluoroRender's default margin
    assert torch.allclose(c.grad, gc, rtol=1e-3, atol=1e-6 * float(gc.abs().max()))
    assert abs(float(s.grad) - float(gs)) <= 1e-3 * abs(float(gs))


def test_sigma_s_gradient_against_central_differences_with_common_random_numbers():
    """For a linear functional L = sum(adj * I) both the adjoint (frozen sampling) and a central
    difference of re-rendered films with the same paths (step 5 % of sigma_s) are unbiased for
    dE[L]/dsigma_s (the difference up to O(h^2)); compared over paired batches of paths. (For a
    quadratic loss they are not comparable: each would also differentiate its own variance.)"""
    sc = adjoint_scene(n_paths=1)
    S = Scene(sc)
    conc = torch.from_numpy(sc["medium"]["conc"]).cuda()
    rng = np.random.default_rng(8)
    adj = torch.from_numpy((1.0 + 0.5 * rng.normal(size=(12, 12, sg.N_BINS))).astype(np.float32)
                           ).cuda()
    K, n, s0 = 8, 100_000, 10.0
    h = 0.05 * s0
    diffs, grads = [], []
    for k in range(K):
        def L(sig):
            S.set_medium_values(conc, sig)
            f = S.render(form="wavefront", n_paths=n, path_offset=k * n)
            return float((f.double() * adj.double()).sum())
        fd = (L(s0 + h) - L(s0 - h)) / (2 * h)
        S.set_medium_values(conc, s0)
        gs = torch.zeros(1, device="cuda")
        S.adjoint(adj, None, gs, n_paths=n, path_offset=k * n, majorant_margin=0.1)
        grads.append(float(gs))
        diffs.append(fd - float(gs))
    md, sd = batch_mean_se(diffs)
    mg = float(np.mean(grads))
    assert abs(md) <= 3 * sd + 0.02 * abs(mg), (md, sd, mg)
    assert abs(mg) > 3 * batch_mean_se(grads)[1]


def test_adjoint_full_size_linearity_and_finiteness():
    """The 64^3 x 2 dyes / 256x256 / 32 spp workload: gradients are finite and linear in the
    adjoint film (a property that holds at any size)."""
    sc = sg.cfg4_adjoint()
    S = Scene(sc)
    n = sc["params"]["n_paths"]
    rng = np.random.default_rng(1)
    a1 = torch.from_numpy(rng.normal(size=(256, 256, sg.N_BINS)).astype(np.float32)).cuda()
    a2 = torch.from_numpy(rng.normal(size=(256, 256, sg.N_BINS)).astype(np.float32)).cuda()
    out = []
    for adj in (a1, a2, a1 + 2.0 * a2):
        gc = torch.zeros(S.conc_t.shape, device="cuda")
        gs = torch.zeros(1, device="cuda")
        S.adjoint(adj, gc, gs, n_paths=n, majorant_margin=0.1)
        out.append((gc.double(), float(gs)))
    assert all(torch.isfinite(o[0]).all() for o in out)
    comb = out[0][0] + 2.0 * out[1][0]
    scale = float(comb.abs().max())
    assert scale > 0
    assert torch.allclose(out[2][0], comb, rtol=1e-3, atol=1e-4 * scale)
    assert abs(out[2][1] - (out[0][1] + 2 * out[1][1])) <= 1e-3 * (abs(out[0][1]) + 2 * abs(out[1][1]))


def test_cfg4_gradient_against_frozen_central_differences_on_64_voxels():
    """Config 4 at full size (2 x 64^3 blob dyes, sigma_s 30, 256 x 256 x 81 ortho film, 32 paths
    per pixel): the gradient of the L2 loss sum (I - T)^2 against a seeded target T, taken by
    flr_adjoint at theta_0 as the gradient of the linear functional sum(adj I) with
    adj = 2 (I(theta_0) - T), against central differences with a step of 1e-3 of the value, common
    random numbers (same seed and path ids) and the frozen-sampling estimator
    (flr_debug_frozen_sums), on 64 seeded random voxels (c >= 0.05) and sigma_s. Eight disjoint path
    batches give an adjoint and a difference per batch. The frozen estimator's derivative is the
    score-function estimator flr_adjoint evaluates (Eq. 6 for the transmittance terms), so the two
    agree path by path up to O(h^2) and fp32 rounding:
      - each voxel passes if the mean difference is within max(3 SE, 1 % of the gradient) (plus
        1e-6 of the largest, for gradients near zero);
      - sigma_s enters every null and scattering decision and every transmittance of a path, and a
        batch's sigma_s gradient is a few per cent of the sum of its paths' |derivatives| (a few
        heavy paths of both signs carry it), so the per-path agreement is checked directly on the
        heaviest paths (single-path replays, within 2e-3), and the batches against it: the mean
        difference within max(3 SE, 1 % of the gradient, 1e-3 of the mean sum over paths of
        |derivative|). The sigma_s difference is Richardson's combination (4 D(h/2) - D(h)) / 3 of
        the steps 1e-3 and 5e-4 (the O(h^2) term of many decisions per path)."""
    sc = sg.cfg4_adjoint(field_seed=0, seed=0)
    n = sc["params"]["n_paths"]
    assert n == 256 * 256 * 32 and sc["medium"]["conc"].shape == (2, 64, 64, 64)
    mg = 0.1
    S = Scene(sc)
    target = Scene(sg.cfg4_adjoint(field_seed=1, seed=1000)).render(form="wavefront_warp").clone()
    film = S.render(form="wavefront_warp", majorant_margin=mg)
    adj = (2.0 * (film - target)).float().contiguous()
    conc = sc["medium"]["conc"]
    rng = np.random.default_rng(64)
    cand = np.argwhere(conc >= 0.05)
    pick = cand[rng.choice(cand.shape[0], size=64, replace=False)]
    nz, ny, nx = conc.shape[1:]
    voxels = [(int(d), int((z * ny + y) * nx + x), float(conc[d, z, y, x])) for d, z, y, x in pick]
    s0 = float(sc["medium"]["sigma_s"])
    hs = 1e-3 * s0
    K = 8
    m = n // K
    fd = np.zeros((K, 65))
    ad = np.zeros((K, 65))
    abs_sum = np.zeros(K)
    heavy = None
    for k in range(K):
        gc = torch.zeros(S.conc_t.shape, dtype=torch.float32, device="cuda")
        gs = torch.zeros(1, dtype=torch.float32, device="cuda")
        S.adjoint(adj, gc, gs, n_paths=m, path_offset=k * m, majorant_margin=mg)
        g = gc.double().cpu().numpy().reshape(2, -1)
        for j, (d, v, c0) in enumerate(voxels):
            h = 1e-3 * c0
            sp = S.frozen_sums(adj, (d, v, h, 0.0), n_paths=m, path_offset=k * m, majorant_margin=mg)
            sm = S.frozen_sums(adj, (d, v, -h, 0.0), n_paths=m, path_offset=k * m, majorant_margin=mg)
            fd[k, j] = float((sp - sm).sum()) / (2 * h)
            ad[k, j] = g[d, v]

        def cdiff(h):
            sp = S.frozen_sums(adj, (-1, 0, 0.0, h), n_paths=m, path_offset=k * m, majorant_margin=mg)
            sm = S.frozen_sums(adj, (-1, 0, 0.0, -h), n_paths=m, path_offset=k * m, majorant_margin=mg)
            return (sp - sm) / (2 * h)
        d1, d2 = cdiff(hs), cdiff(hs / 2)
        per_path = (4.0 * d2 - d1) / 3.0
        fd[k, 64] = float(per_path.sum())
        ad[k, 64] = float(gs.item())
        abs_sum[k] = float(per_path.abs().sum())
        if k == 0:
            heavy = torch.argsort(per_path.abs(), descending=True)[:16].cpu().numpy()
    assert S.status() == N.FLR_OK
    ma, sa = batch_mean_se(ad)
    md, sd = batch_mean_se(fd - ad)
    scale = np.abs(ma[:64]).max()
    tol = np.maximum(3 * sd, 1e-2 * np.abs(ma))
    tol[:64] += 1e-6 * scale
    tol[64] = max(tol[64], 1e-3 * abs_sum.mean())
    bad = np.where(np.abs(md) > tol)[0]
    assert bad.size == 0, [(int(j), ma[j], md[j], sd[j], tol[j]) for j in bad]
    # not a comparison of zeros: most chosen voxels lie on some path's decisions or marches, and
    # over them the differences are small against the gradients themselves (the per-voxel
    # gradients of one 2.1M-path estimate are heavy-tailed, so they are not all resolved from zero)
    nonzero = np.abs(ma[:64]) > 0
    assert int(nonzero.sum()) >= 32, int(nonzero.sum())
    assert np.abs(md[:64][nonzero]).sum() <= 1e-2 * np.abs(ma[:64][nonzero]).sum()
    assert ma[64] != 0.0
    # the heaviest paths one by one (a one-path launch: both sides scale by 1 instead of 1/m)
    gc1 = torch.zeros(S.conc_t.shape, dtype=torch.float32, device="cuda")
    gs1 = torch.zeros(1, dtype=torch.float32, device="cuda")
    for i in heavy:
        i = int(i)
        S.adjoint(adj, gc1, gs1, n_paths=1, path_offset=i, majorant_margin=mg, form="plain")
        a1 = float(gs1.item())
        one = []
        for h in (hs, hs / 2):
            sp = float(S.frozen_sums(adj, (-1, 0, 0.0, h), n_paths=1, path_offset=i, majorant_margin=mg)[0])
            sm = float(S.frozen_sums(adj, (-1, 0, 0.0, -h), n_paths=1, path_offset=i, majorant_margin=mg)[0])
            one.append((sp - sm) / (2 * h))
        f1 = (4.0 * one[1] - one[0]) / 3.0
        assert abs(f1 - a1) <= 2e-3 * abs(a1) + 1e-12, (i, f1, a1)
