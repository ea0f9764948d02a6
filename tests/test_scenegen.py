"""The seeded input generators reproduce the stated workloads: sizes, spectra, coefficients and
path counts of the five configurations, and the same arrays on every call (inputs never drift
between the oracle and the GPU, or between runs). No method arithmetic is tested here."""
import math

import numpy as np

import scenegen as sg


def _same(a, b):
    if isinstance(a, dict):
        return a.keys() == b.keys() and all(_same(a[k], b[k]) for k in a)
    if isinstance(a, (list, tuple)):
        return len(a) == len(b) and all(_same(x, y) for x, y in zip(a, b))
    if isinstance(a, np.ndarray):
        return np.array_equal(a, b)
    return a == b


def bins(lam):
    return int(math.ceil((lam - sg.LAMBDA0) / sg.DLAMBDA - 0.5))


def test_spectrum_grid():
    sp = sg.spectrum()
    assert (sp["n_bins"], sp["lambda0"], sp["dlambda"]) == (81, 380.0, 5.0)
    c = sg.bin_centres()
    assert c[0] == 380.0 and c[-1] == 780.0


def test_homogeneous_cube():
    sc = sg.cfg1_homogeneous_cube()
    assert sc["params"]["n_paths"] == 100_000 and sc["params"]["seed"] == 0
    assert sc["params"]["n_rr"] == 5
    d = sc["dyes"]
    a, e = d["abs_shape"][0], d["emit_spec"][0]
    assert np.argmax(a) == bins(490.0) and a.max() == 1.0
    assert np.argmax(e) == bins(520.0)
    assert float(d["eps"][0]) == 2.0 and abs(float(d["qy"][0]) - 0.9) < 1e-7
    assert sc["medium"]["sigma_s"] == 20.0
    assert (sc["sensor"]["width"], sc["sensor"]["height"]) == (64, 64)
    assert _same(sc, sg.cfg1_homogeneous_cube())


def test_cornell_box():
    sc = sg.cfg2_cornell_box()
    assert sc["params"]["n_paths"] == 512 * 512 * 16
    conc = sc["medium"]["conc"]
    assert conc.shape == (4, 128, 128, 128) and conc.dtype == np.float32
    assert sc["medium"]["sigma_s"] == 50.0
    em = [int(np.argmax(sc["dyes"]["emit_spec"][d])) for d in range(4)]
    assert em == [bins(450.0), bins(520.0), bins(600.0), bins(680.0)]
    qy = sc["dyes"]["qy"]
    assert (qy >= 0.3).all() and (qy <= 0.95).all()
    assert (sc["sensor"]["kind"], sc["sensor"]["width"], sc["sensor"]["height"]) == ("pinhole", 512, 512)
    lines = sc["sources"][0]["lines_nm"]
    assert len(sc["sources"]) == 1 and len(lines) == 4
    # each sphere is one dye's, and each dye fills a sphere of radius 0.15-0.25 of the box
    occupied = (conc > 0).reshape(4, -1)
    assert not (occupied.sum(axis=0) > 1).any()
    r = np.cbrt(occupied.sum(axis=1) / 128 ** 3 * 3 / (4 * math.pi))
    assert ((r > 0.14) & (r < 0.26)).all(), r
    assert _same(sc, sg.cfg2_cornell_box())


def test_batched_media():
    media = sg.cfg3_batched_media()
    assert len(media) == 256
    n = np.array([m["params"]["n_paths"] for m in media])
    assert n.min() >= 10_000 and n.max() <= 1_000_000
    assert 3e7 < n.sum() < 8e7
    edges, dyes = [], []
    for m in media:
        c = m["medium"].get("conc")
        if c is not None:
            edges.append(c.shape[-1])
            assert c.shape[-1] == c.shape[-2] == c.shape[-3]
        dyes.append(m["dyes"]["eps"].shape[0])
    assert min(edges) >= 16 and max(edges) <= 128
    assert set(dyes) <= {1, 2, 3} and len(set(dyes)) == 3
    assert _same(media[:3], sg.cfg3_batched_media()[:3])


def test_adjoint_workload():
    sc = sg.cfg4_adjoint()
    assert sc["params"]["n_paths"] == 256 * 256 * 32
    assert sc["medium"]["conc"].shape == (2, 64, 64, 64)
    assert sc["medium"]["sigma_s"] == 30.0
    assert (sc["sensor"]["kind"], sc["sensor"]["width"]) == ("ortho", 256)
    t = sg.cfg4_adjoint(field_seed=1)
    assert not np.array_equal(sc["medium"]["conc"], t["medium"]["conc"])
    assert _same(sc, sg.cfg4_adjoint())


def test_light_sheet():
    sc = sg.cfg5_light_sheet()
    assert sc["params"]["n_paths"] == 1024 * 1024 * 64
    assert sc["medium"]["conc"].shape == (4, 256, 256, 256)
    assert (sc["sensor"]["kind"], sc["sensor"]["width"], sc["sensor"]["height"]) == ("ortho", 1024, 1024)
    src = sc["sources"][0]
    assert src["lines_nm"] == [488.0] and bins(488.0) == 22
    # albedo 0.999 at the source line: sigma_s / (sigma_s + sum_d eps_d a_d(490) mean c_d)
    d = sc["dyes"]
    conc = sc["medium"]["conc"].reshape(4, -1).astype(np.float64)
    sig_a = float((d["eps"].astype(np.float64) * d["abs_shape"][:, 22] * conc.mean(axis=1)).sum())
    s = sc["medium"]["sigma_s"]
    assert abs(s / (s + sig_a) - 0.999) < 1e-4
    assert _same(sc["dyes"], sg.cfg5_light_sheet()["dyes"])
