"""Pins for the oracle's forward model f (Eq. 3) and per-ray decomposition UDM (Eq. 13)."""
import numpy as np
import pytest

from oracle import spectral
from synth import spectra


class _Mono:
    """Two monochromatic spectra (one energy bin each): f becomes linear in a."""

    def __init__(self, e_h=90.0, e_l=50.0, e_ref=60.0):
        e = np.array([e_l, e_h])
        self.energy_kev = e
        self.s_high = np.array([0.0, 1.0])
        self.s_low = np.array([1.0, 0.0])
        self.f_kn = spectra.klein_nishina(e)
        self.f_p = spectra.photoelectric(e, e_ref)


def test_f_of_zero_is_zero():
    t = spectra.SpectralTables()
    fh, fl = spectral.forward_model(t, np.zeros(3), np.zeros(3))
    assert np.all(np.abs(fh) < 1e-15) and np.all(np.abs(fl) < 1e-15)


def test_monochromatic_forward_model_is_linear():
    s = _Mono()
    rng = np.random.default_rng(0)
    ac, ap = rng.uniform(0, 5, 20), rng.uniform(0, 2, 20)
    fh, fl, J = spectral.forward_model(s, ac, ap, jacobian=True)
    assert np.allclose(fh, s.f_kn[1] * ac + s.f_p[1] * ap, rtol=1e-13)
    assert np.allclose(fl, s.f_kn[0] * ac + s.f_p[0] * ap, rtol=1e-13)
    assert np.allclose(J, [[s.f_kn[1], s.f_p[1], s.f_kn[0], s.f_p[0]]] * 20, rtol=1e-13)


def test_polychromatic_beam_hardening_is_concave():
    # f is concave along a ray (beam hardening): f(2a) < 2 f(a) for a > 0
    t = spectra.SpectralTables(e_ref_kev=100.0)
    a = np.array([1.0, 3.0, 8.0])
    f1 = spectral.forward_model(t, a, 0.1 * a)[0]
    f2 = spectral.forward_model(t, 2 * a, 0.2 * a)[0]
    assert np.all(f2 < 2 * f1)


@pytest.mark.parametrize("e_ref", [1.0, 100.0])
def test_jacobian_matches_central_differences(e_ref):
    t = spectra.SpectralTables(e_ref_kev=e_ref)
    rng = np.random.default_rng(1)
    ac = rng.uniform(0.1, 10, 30)
    ap = rng.uniform(0.0, 1.0, 30) * (1e3 if e_ref == 1.0 else 1.0)
    _, _, J = spectral.forward_model(t, ac, ap, jacobian=True)
    for j, (dc, dp) in enumerate([(1, 0), (0, 1)]):
        h = 1e-5 if dc else 1e-5 * max(1.0, ap.max())
        fhp, flp = spectral.forward_model(t, ac + h * dc, ap + h * dp)
        fhm, flm = spectral.forward_model(t, ac - h * dc, ap - h * dp)
        assert np.allclose((fhp - fhm) / (2 * h), J[:, j], rtol=1e-7, atol=1e-14)
        assert np.allclose((flp - flm) / (2 * h), J[:, 2 + j], rtol=1e-7, atol=1e-14)


def _ones(n):
    return np.ones(n)


def test_monochromatic_udm_with_zero_rho_is_a_2x2_linear_solve():
    s = _Mono()
    rng = np.random.default_rng(2)
    n = 50
    true_c, true_p = rng.uniform(0, 6, n), rng.uniform(0, 3, n)
    A = np.array([[s.f_kn[1], s.f_p[1]], [s.f_kn[0], s.f_p[0]]])
    m = A @ np.stack([true_c, true_p])
    # weights change nothing when the system is square and exactly solvable
    wh, wl = rng.uniform(1, 10, n), rng.uniform(1, 10, n)
    ac, ap, mu, st = spectral.udm(s, m[0], m[1], wh, wl, np.zeros(n), np.zeros(n), 0.0, 0.0, 40,
                                  np.zeros(n), np.zeros(n), np.full(n, 1e-3))
    sol = np.linalg.solve(A, m)
    assert np.allclose(ac, sol[0], atol=1e-9) and np.allclose(ap, sol[1], atol=1e-9)


def test_monochromatic_udm_with_rho_is_a_regularised_linear_solve():
    # Eq. 13 with linear f: (A^T W A + diag rho) a = A^T W m + rho v
    s = _Mono()
    rng = np.random.default_rng(3)
    n = 20
    m = rng.uniform(0.5, 3.0, (2, n))
    wh, wl = rng.uniform(1, 10, n), rng.uniform(1, 10, n)
    vc, vp = rng.uniform(0, 2, n), rng.uniform(0, 2, n)
    rho = (0.7, 2.5)
    ac, ap, _, _ = spectral.udm(s, m[0], m[1], wh, wl, vc, vp, rho[0], rho[1], 60,
                                np.zeros(n), np.zeros(n), np.full(n, 1e-3))
    A = np.array([[s.f_kn[1], s.f_p[1]], [s.f_kn[0], s.f_p[0]]])
    for r in range(n):
        W = np.diag([wh[r], wl[r]])
        lhs = A.T @ W @ A + np.diag(rho)
        rhs = A.T @ W @ m[:, r] + np.array(rho) * np.array([vc[r], vp[r]])
        sol = np.linalg.solve(lhs, rhs)
        assert ac[r] == pytest.approx(sol[0], abs=1e-9) and ap[r] == pytest.approx(sol[1], abs=1e-9)


def test_noise_free_polychromatic_recovers_line_integrals():
    # PE made identifiable with E_ref = 100 keV; rho = 0, unit weights, exact data
    t = spectra.SpectralTables(e_ref_kev=100.0)
    rng = np.random.default_rng(4)
    n = 40
    true_c, true_p = rng.uniform(0.5, 8, n), rng.uniform(0.0, 1.5, n)
    # the data are made here from the definition of Eq. 2 (not with the oracle's f)
    att = np.exp(-np.outer(true_c, t.f_kn) - np.outer(true_p, t.f_p))
    mh, ml = -np.log(att @ t.s_high), -np.log(att @ t.s_low)
    ac, ap, _, st = spectral.udm(t, mh, ml, _ones(n), _ones(n), np.zeros(n), np.zeros(n), 0.0, 0.0, 60,
                                 mh / t.f_kn.mean(), np.zeros(n), np.full(n, 1e-3))
    assert np.allclose(ac, true_c, atol=1e-7) and np.allclose(ap, true_p, atol=1e-7)


def test_udm_matches_brute_force_grid_search():
    # Eq. 13's minimiser found by exhaustive search of the cost on a grid, then refined grids
    t = spectra.SpectralTables(e_ref_kev=100.0)
    rng = np.random.default_rng(5)
    n = 30
    true_c, true_p = rng.uniform(0.5, 4, n), rng.uniform(0.0, 1.0, n)
    att = np.exp(-np.outer(true_c, t.f_kn) - np.outer(true_p, t.f_p))
    mh = -np.log(att @ t.s_high) + rng.normal(0, 0.01, n)
    ml = -np.log(att @ t.s_low) + rng.normal(0, 0.01, n)
    wh, wl = rng.uniform(1e3, 1e4, n), rng.uniform(1e3, 1e4, n)
    vc, vp = true_c + rng.normal(0, 0.05, n), true_p + rng.normal(0, 0.05, n)
    rho = (50.0, 200.0)
    ac, ap, _, _ = spectral.udm(t, mh, ml, wh, wl, vc, vp, rho[0], rho[1], 80, vc, vp, np.full(n, 1e-3))
    def grid_cost(r, C, Pp):
        # the cost written out from Eq. 13 with the Eq. 2-3 forward model
        att = np.exp(-np.outer(C.ravel(), t.f_kn) - np.outer(Pp.ravel(), t.f_p))
        fh, fl = -np.log(att @ t.s_high), -np.log(att @ t.s_low)
        return (0.5 * (wh[r] * (fh - mh[r]) ** 2 + wl[r] * (fl - ml[r]) ** 2)
                + 0.5 * rho[0] * (C.ravel() - vc[r]) ** 2 + 0.5 * rho[1] * (Pp.ravel() - vp[r]) ** 2)

    for r in range(n):
        lm_cost = spectral.udm_cost(t, mh[r:r + 1], ml[r:r + 1], wh[r:r + 1], wl[r:r + 1], vc[r:r + 1],
                                    vp[r:r + 1], rho[0], rho[1], ac[r:r + 1], ap[r:r + 1])[0]
        # no point of a wide exhaustive grid beats the LM answer (global basin)
        C, Pp = np.meshgrid(np.linspace(true_c[r] - 0.5, true_c[r] + 0.5, 101),
                            np.linspace(true_p[r] - 0.5, true_p[r] + 0.5, 101))
        assert lm_cost <= grid_cost(r, C, Pp).min() + 1e-12
        # nor does any point of a fine grid around it (local optimality at grid resolution)
        C, Pp = np.meshgrid(np.linspace(ac[r] - 5e-3, ac[r] + 5e-3, 101), np.linspace(ap[r] - 5e-3, ap[r] + 5e-3, 101))
        assert lm_cost <= grid_cost(r, C, Pp).min() + 1e-12


def test_lm_never_increases_cost_and_damping_moves_by_ten():
    t = spectra.SpectralTables()
    rng = np.random.default_rng(6)
    n = 200
    mh, ml = rng.uniform(0.5, 5, n), rng.uniform(0.6, 6, n)
    wh, wl = rng.uniform(1e3, 1e5, n), rng.uniform(1e3, 1e5, n)
    vc, vp = mh * 0.9, rng.uniform(0, 1e-3, n)
    a_c, a_p, mu = mh.copy(), np.zeros(n), np.full(n, 1e-3)
    prev = spectral.udm_cost(t, mh, ml, wh, wl, vc, vp, 1e-3, 1e-3, a_c, a_p)
    for _ in range(6):
        a_c, a_p, mu_new, st = spectral.udm(t, mh, ml, wh, wl, vc, vp, 1e-3, 1e-3, 1, a_c, a_p, mu)
        cost = spectral.udm_cost(t, mh, ml, wh, wl, vc, vp, 1e-3, 1e-3, a_c, a_p)
        assert np.all(cost <= prev)
        acc = st == 0
        assert np.allclose(mu_new[acc], np.maximum(mu[acc] / 10, 1e-10))
        assert np.allclose(mu_new[st == 1], np.minimum(mu[st == 1] * 10, 1e10))
        assert np.all(cost[acc] < prev[acc])
        prev, mu = cost, mu_new
