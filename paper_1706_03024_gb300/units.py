"""Conversions from the spectroscopic quantities the paper's dyes are described by (Sec. 4.1 and
Sec. 5: molar absorptivity, concentration in grams per litre, quantum yield) to the library's
inputs: `eps` of flr_set_dyes is the napierian absorption coefficient, in cm^-1, per unit of the
concentration stored in the grids, at the peak of the dye's (peak-normalised) absorption shape.

Tables of molar absorptivity are decadic: absorbance A = eps_10 * c * l, with eps_10 in
M^-1 cm^-1, c in mol/L and l in cm, and transmittance 10^-A. The napierian coefficient of the same
solution is sigma_a = ln(10) * eps_10 * c in cm^-1 (transmittance exp(-sigma_a l)).
"""
from __future__ import annotations

import math

LN10 = math.log(10.0)


def molarity(grams_per_litre: float, molar_mass: float) -> float:
    """mol/L from g/L and the molar mass in g/mol."""
    if molar_mass <= 0.0:
        raise ValueError("molar mass must be positive")
    return grams_per_litre / molar_mass


def napierian_sigma_a(eps_decadic: float, molar: float) -> float:
    """Absorption coefficient sigma_a in cm^-1 of a solution of `molar` mol/L of a dye with decadic
    molar absorptivity eps_decadic (M^-1 cm^-1)."""
    if eps_decadic < 0.0 or molar < 0.0:
        raise ValueError("molar absorptivity and concentration must be non-negative")
    return LN10 * eps_decadic * molar


def dye_eps(eps_decadic: float, unit_molar: float) -> float:
    """The library's `eps` for a dye whose grid values count concentration in units of
    `unit_molar` mol/L (grid value 1 = unit_molar): the napierian peak coefficient per grid unit."""
    return napierian_sigma_a(eps_decadic, unit_molar)


def brightness(eps_decadic: float, quantum_yield: float) -> float:
    """The brightness of a fluorophore: molar absorptivity times quantum yield (M^-1 cm^-1), the
    quantity that ranks how much fluorescence a dye gives at equal concentration (Sec. 5)."""
    if not 0.0 <= quantum_yield <= 1.0:
        raise ValueError("quantum yield must be in [0, 1]")
    return eps_decadic * quantum_yield
