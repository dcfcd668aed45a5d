"""Pins for the spectral input tables (Eq. 1's f_KN, f_p; the spectra S of Eq. 2)."""
import numpy as np
import pytest
from scipy import integrate

from synth import spectra


def _kn_by_quadrature(e_kev):
    """f_KN from the Klein-Nishina differential cross-section, integrated over angle.

    dsigma/dOmega = r_e^2/2 P^2 (P + 1/P - sin^2 th), P = 1/(1 + alpha(1 - cos th));
    f_KN = sigma / (2 pi r_e^2) = int_0^pi (1/2) P^2 (P + 1/P - sin^2 th) sin th dth.
    """
    alpha = e_kev / spectra.ELECTRON_REST_KEV

    def integrand(th):
        P = 1.0 / (1.0 + alpha * (1.0 - np.cos(th)))
        return 0.5 * P * P * (P + 1.0 / P - np.sin(th) ** 2) * np.sin(th)

    val, _ = integrate.quad(integrand, 0.0, np.pi, epsabs=1e-14, epsrel=1e-13)
    return val


@pytest.mark.parametrize("e", [20.0, 45.5, 60.0, 100.0, 140.0, 511.0, 2000.0])
def test_klein_nishina_matches_angular_integral(e):
    assert spectra.klein_nishina(np.array([e]))[0] == pytest.approx(_kn_by_quadrature(e), rel=1e-10)


def test_klein_nishina_thomson_limit():
    # sigma_KN -> sigma_Thomson = (8 pi / 3) r_e^2, i.e. f_KN -> 4/3; the low-energy series is
    # sigma/sigma_T = 1 - 2a + 26/5 a^2 - 133/10 a^3 + O(a^4)
    a = 2e-3
    e = a * spectra.ELECTRON_REST_KEV
    series = 4.0 / 3.0 * (1.0 - 2.0 * a + 26.0 / 5.0 * a * a - 133.0 / 10.0 * a**3)
    assert spectra.klein_nishina(np.array([e]))[0] == pytest.approx(series, rel=1e-7)


def test_klein_nishina_textbook_value_at_511kev():
    # sigma_KN(511 keV) / sigma_Thomson = 0.4307 (standard tabulated value)
    ratio = spectra.klein_nishina(np.array([spectra.ELECTRON_REST_KEV]))[0] * 0.75
    assert ratio == pytest.approx(0.4307, abs=2e-4)


def test_klein_nishina_monotone_decreasing_on_grid():
    f = spectra.klein_nishina(spectra.energy_grid())
    assert np.all(np.diff(f) < 0)


def test_photoelectric_cubic():
    e = spectra.energy_grid()
    f = spectra.photoelectric(e, 1.0)
    assert np.allclose(f * e**3, 1.0, rtol=1e-14)
    assert spectra.photoelectric(np.array([50.0]), 100.0)[0] == pytest.approx(8.0)


def test_grid_and_spectra():
    e = spectra.energy_grid()
    assert e.size == 121 and e[0] == 20.0 and e[-1] == 140.0
    t = spectra.SpectralTables()
    for s in (t.s_high, t.s_low):
        assert s.sum() == pytest.approx(1.0, abs=1e-14)
        assert np.all(s >= 0)
    assert np.all(t.s_low[e >= 80.0] == 0) and np.all(t.s_low[e < 80.0] > 0)
    assert np.all(t.s_high[e >= 140.0] == 0) and np.all(t.s_high[e < 140.0] > 0)
    # the filtered low spectrum is softer: its mean energy is below the high one's
    assert np.dot(t.s_low, e) < np.dot(t.s_high, e)


def test_unfiltered_kramers_shape():
    e = spectra.energy_grid()
    k = spectra.kramers(e, 80.0)
    assert k[e == 40.0][0] == pytest.approx(1.0)  # (80-40)/40
    assert k[e == 79.0][0] == pytest.approx(1.0 / 79.0)


def test_aluminium_compton_attenuation_scale():
    # electron density of Al (7.83e23 cm^-3) times 2 pi r_e^2 f_KN: ~0.39 f_KN cm^-1
    mu = spectra.aluminium_mu(np.array([60.0]))[0]
    f = spectra.klein_nishina(np.array([60.0]))[0]
    assert mu / f == pytest.approx(0.3907, rel=2e-3)
