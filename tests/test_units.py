"""Unit conversions of the dye description (decadic molar absorptivity, g/L) into the library's
napierian per-unit-concentration `eps`, checked against their definitions: a solution's decadic
absorbance A = eps_10 c l transmits 10^-A, which the napierian coefficient must reproduce as
exp(-sigma_a l); and with that `eps` the oracle's non-scattering slab transmits 10^-A."""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg
from paper_1706_03024_gb300 import units
from tests.stats import binomial_se


def test_napierian_coefficient_reproduces_decadic_transmittance():
    for eps10, molar, length in ((73000.0, 1e-6, 1.0), (5000.0, 2e-5, 0.5), (1.0, 0.3, 2.0)):
        a = eps10 * molar * length
        s = units.napierian_sigma_a(eps10, molar)
        assert math.exp(-s * length) == pytest.approx(10.0 ** (-a), rel=1e-12)


def test_grams_per_litre_and_grid_units():
    assert units.molarity(10.0, 500.0) == pytest.approx(0.02)
    # a grid value 2.0 in units of 1 uM is 2 uM
    e = units.dye_eps(40000.0, 1e-6)
    assert 2.0 * e == pytest.approx(units.napierian_sigma_a(40000.0, 2e-6))
    assert units.brightness(40000.0, 0.5) == 20000.0
    for bad in ((lambda: units.molarity(1.0, 0.0)), (lambda: units.napierian_sigma_a(-1.0, 1.0)),
                (lambda: units.brightness(1.0, 1.5))):
        with pytest.raises(ValueError):
            bad()


def test_slab_of_converted_dye_transmits_decadic_absorbance():
    """A 1 cm cube of a non-emitting dye at its absorption peak (Eq. 6 in the library's units)."""
    eps10, molar = 30000.0, 1.5e-5          # absorbance 0.45 over 1 cm
    eps = units.dye_eps(eps10, 1e-6)        # grid values in uM
    dyes = sg.make_dyes([490.0], [15.0], [620.0], [15.0], eps=[eps], qy=[0.0])
    sc = {"spectrum": sg.spectrum(), "dyes": dyes,
          "medium": sg.homogeneous_medium(1, conc=molar / 1e-6, sigma_s=0.0),
          "sources": [sg.pencil_beam((0.5, 0.5, 1.0), (0, 0, -1), [490.0])],
          "sensor": sg.no_sensor(), "params": sg.params(200_000, seed=1)}
    r = oracle.render(sc)
    T = r["face"][0, sg.FACE_NZ].sum()
    want = 10.0 ** (-eps10 * molar)
    assert abs(T - want) <= 3 * binomial_se(want, 200_000), (T, want)
    assert float(np.float32(eps)) > 0
