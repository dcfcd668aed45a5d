"""Spectral input tables for the two-basis attenuation model (Eq. 1, Eq. 2).

The paper takes the Compton and photoelectric energy dependences f_KN(E), f_p(E)
and the two source spectra S_h(E), S_l(E) as given (Sec. 1, the footnote to
Eq. 1 defers their definition to the constrained-decomposition paper it cites).
This module tabulates them on a discrete energy grid; the reconstruction only
ever receives the tables.

Readings used here:
  * f_KN: the Klein-Nishina total cross-section divided by 2*pi*r_e^2, in the
    Alvarez-Macovski normalisation, of alpha = E / (m_e c^2). It tends to 4/3
    as alpha -> 0 (Thomson limit).
  * f_p: (E_ref / E)^3, "cubic decay with E" (Sec. 1); E_ref is a parameter.
  * S: Kramers' photon-number spectrum (kVp - E) / E below kVp, filtered by
    2 mm of aluminium whose attenuation is the Compton part only
    (electron density of Al times the Klein-Nishina cross-section) plus an
    optional k_al * E^-3 photoelectric term (default 0).
  * The integral over E becomes a sum over 1 keV bins.
"""
from __future__ import annotations

import numpy as np

ELECTRON_REST_KEV = 510.99895  # m_e c^2, CODATA 2018
CLASSICAL_ELECTRON_RADIUS_CM = 2.8179403262e-13  # r_e, CODATA 2018
AVOGADRO = 6.02214076e23
AL_DENSITY_G_CM3 = 2.699
AL_Z = 13.0
AL_A_G_MOL = 26.9815385


def energy_grid(e_min_kev: float = 20.0, e_max_kev: float = 140.0, step_kev: float = 1.0) -> np.ndarray:
    """Energies of the spectral bins, inclusive of both ends (20..140 keV -> 121 samples)."""
    n = int(round((e_max_kev - e_min_kev) / step_kev)) + 1
    return e_min_kev + step_kev * np.arange(n, dtype=np.float64)


def klein_nishina(e_kev: np.ndarray) -> np.ndarray:
    """f_KN(E): Klein-Nishina total cross-section / (2 pi r_e^2).

    f = (1+a)/a^2 [2(1+a)/(1+2a) - ln(1+2a)/a] + ln(1+2a)/(2a) - (1+3a)/(1+2a)^2,
    a = E / 510.999 keV. Evaluated in FP64; cancellation makes it inaccurate
    below a ~ 1e-3 (E < 0.5 keV), far below the 20 keV grid floor.
    """
    a = np.asarray(e_kev, dtype=np.float64) / ELECTRON_REST_KEV
    l = np.log1p(2.0 * a)
    t1 = (1.0 + a) / a**2 * (2.0 * (1.0 + a) / (1.0 + 2.0 * a) - l / a)
    t2 = l / (2.0 * a)
    t3 = (1.0 + 3.0 * a) / (1.0 + 2.0 * a) ** 2
    return t1 + t2 - t3


def photoelectric(e_kev: np.ndarray, e_ref_kev: float = 1.0) -> np.ndarray:
    """f_p(E) = (E_ref / E)^3."""
    return (e_ref_kev / np.asarray(e_kev, dtype=np.float64)) ** 3


def aluminium_mu(e_kev: np.ndarray, k_al: float = 0.0) -> np.ndarray:
    """Linear attenuation of Al (cm^-1): Compton part from its electron density, plus k_al E^-3."""
    n_e = AL_DENSITY_G_CM3 * AVOGADRO * AL_Z / AL_A_G_MOL  # electrons / cm^3
    sigma0 = 2.0 * np.pi * CLASSICAL_ELECTRON_RADIUS_CM**2  # cm^2
    e = np.asarray(e_kev, dtype=np.float64)
    return n_e * sigma0 * klein_nishina(e) + k_al * e**-3


def kramers(e_kev: np.ndarray, kvp: float) -> np.ndarray:
    """Kramers' photon-number spectrum (kVp - E)/E for E < kVp, else 0 (unnormalised)."""
    e = np.asarray(e_kev, dtype=np.float64)
    return np.where(e < kvp, (kvp - e) / e, 0.0)


def source_spectrum(e_kev: np.ndarray, kvp: float, al_mm: float = 2.0, k_al: float = 0.0) -> np.ndarray:
    """Filtered Kramers spectrum normalised to unit sum over the grid."""
    s = kramers(e_kev, kvp) * np.exp(-aluminium_mu(e_kev, k_al) * (al_mm / 10.0))
    return s / s.sum()


class SpectralTables:
    """The four FP64 tables the method consumes, on one energy grid."""

    def __init__(self, kvp_high: float = 140.0, kvp_low: float = 80.0, al_mm: float = 2.0,
                 e_ref_kev: float = 1.0, k_al: float = 0.0, e_min_kev: float = 20.0,
                 e_max_kev: float = 140.0, step_kev: float = 1.0):
        self.energy_kev = energy_grid(e_min_kev, e_max_kev, step_kev)
        self.s_high = source_spectrum(self.energy_kev, kvp_high, al_mm, k_al)
        self.s_low = source_spectrum(self.energy_kev, kvp_low, al_mm, k_al)
        self.f_kn = klein_nishina(self.energy_kev)
        self.f_p = photoelectric(self.energy_kev, e_ref_kev)
        self.e_ref_kev = e_ref_kev

    @property
    def n_energies(self) -> int:
        return int(self.energy_kev.size)

    def as_dict(self) -> dict:
        return {"S_h": self.s_high, "S_l": self.s_low, "f_kn": self.f_kn, "f_p": self.f_p}
