"""Pins for the oracle's FBP and CDM-FBP (the comparison method of Sec. 4, readings in oracle/fbp.py)."""
import math

import numpy as np
import pytest

from oracle import fbp
from synth import geometry as G
from synth import phantom as P
from synth import spectra


def _disk(cx, cy, r, compton, pe=0.0):
    one = lambda v: np.array([v], dtype=np.float64)
    return P.Phantom(shape=np.array([P.ELLIPSE]), cx=one(cx), cy=one(cy), a=one(r), b=one(r), phi=one(0.0),
                     compton=one(compton), pe=one(pe))


def _radius_map(geom, cx, cy):
    ii, jj = np.meshgrid(np.arange(geom.nx), np.arange(geom.ny))
    X = (ii - 0.5 * (geom.nx - 1)) * geom.pixel_cm
    Y = (jj - 0.5 * (geom.ny - 1)) * geom.pixel_cm
    return np.hypot(X - cx, Y - cy)


@pytest.mark.parametrize("w", [0.05, 0.5, 1.0, 2.0, 3.1])
def test_ramp_kernel_frequency_response_is_the_ramp(w):
    # sum_m h(m) e^{-i w m} for the band-limited kernel (alpha = 1) is |w| / (2 pi) on [-pi, pi]:
    # 1/4 - (2/pi^2) sum_{odd m > 0} cos(m w)/m^2 with sum_{odd m} cos(m w)/m^2 = pi^2/8 (1 - 2|w|/pi)
    n = 20001
    h = fbp.ramp_kernel(n, 1.0)
    m = np.arange(-(n - 1), n)
    assert np.sum(h * np.cos(w * m)) == pytest.approx(w / (2 * math.pi), abs=1e-5)
    # pitch alpha scales the kernel by 1 / alpha^2 (the response in cycles per cm stays |nu|)
    assert np.allclose(fbp.ramp_kernel(7, 0.25), fbp.ramp_kernel(7, 1.0) / 0.0625)


def test_filter_is_a_linear_convolution():
    rng = np.random.default_rng(0)
    p = rng.normal(size=(3, 17))
    Q = fbp.filter_rows(p, 0.3)
    h = fbp.ramp_kernel(17, 0.3)
    for v in range(3):
        full = 0.3 * np.convolve(p[v], h)   # index n + 16 of the full convolution is output bin n
        assert np.allclose(Q[v], full[16:33], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind", ["parallel", "parallel_2pi", "fan"])
def test_disk_is_reconstructed_and_refines(kind):
    errs = []
    for scale in (1, 2):
        n = 64 * scale
        if kind == "parallel":
            g = G.parallel_geometry(n, 180 * scale, 128 * scale, 0.1 / scale, 0.1 / scale)
            ph = _disk(0.4, -0.3, 2.0, 1.0)
        elif kind == "parallel_2pi":
            g = G.parallel_geometry(n, 360 * scale, 128 * scale, 0.1 / scale, 0.1 / scale, span_rad=2 * math.pi)
            ph = _disk(-0.5, 0.7, 1.8, 0.5)
        else:
            g = G.fan_geometry(n, 360 * scale, 128 * scale)
            ph = _disk(4.0, -3.0, 12.0, 1.0)
        lc, _ = P.line_integrals(ph, g)
        x = fbp.fbp(g, lc)
        truth, _ = P.truth_image(ph, g)
        r = _radius_map(g, ph.cx[0], ph.cy[0])
        # outside the disk, within the image's inscribed circle (the ramp's tails do not cancel at the
        # corners of a coarse fan scan)
        inscribed = _radius_map(g, 0.0, 0.0) < 0.5 * g.nx * g.pixel_cm
        inner, outer = r < 0.8 * ph.a[0], (r > 1.3 * ph.a[0]) & inscribed
        val = ph.compton[0]
        # off-centre disk: a mirrored or rotated reconstruction, a missing distance weight or a wrong
        # filter gain all move the interior by far more than this
        assert np.abs(x[inner] - val).max() < 0.01 * val
        assert abs(x[inner].mean() - val) < 5e-4 * val
        assert np.abs(x[outer]).max() < 0.08 * val
        errs.append(np.linalg.norm(x - truth) / np.linalg.norm(truth))
    assert errs[1] < 0.8 * errs[0]


def test_fan_and_parallel_reconstruct_the_same_object():
    ph = _disk(3.0, 5.0, 8.0, 0.3)
    gp = G.parallel_geometry(128, 360, 384, 0.4, 0.2)
    gf = G.fan_geometry(128, 720, 384)
    xp = fbp.fbp(gp, P.line_integrals(ph, gp)[0])
    xf = fbp.fbp(gf, P.line_integrals(ph, gf)[0])
    r = _radius_map(gp, 3.0, 5.0)
    inner = r < 0.8 * 8.0
    assert np.abs(xp[inner] - xf[inner]).max() < 0.01 * 0.3


def test_short_scans_are_rejected():
    with pytest.raises(ValueError):
        fbp.fbp(G.parallel_geometry(8, 9, 12, 0.1, 0.1, span_rad=0.75 * math.pi), np.zeros((9, 12)))
    g = G.Geometry(G.FAN_FLAT, 8, 8, 0.1, 9, 0.0, math.pi, 12, 0.1, 0.0, 5.0, 9.0)
    with pytest.raises(ValueError):
        fbp.fbp(g, np.zeros((9, 12)))


class _Mono:
    """Two monochromatic spectra: f is linear in a (f_k = f_KN(E_k) a_c + f_p(E_k) a_p)."""

    def __init__(self):
        e = np.array([50.0, 90.0])
        self.energy_kev = e
        self.s_high = np.array([0.0, 1.0])
        self.s_low = np.array([1.0, 0.0])
        self.f_kn = spectra.klein_nishina(e)
        self.f_p = spectra.photoelectric(e, 60.0)


def test_cdm_recovers_noise_free_line_integrals_and_clamps_negatives():
    s = _Mono()
    rng = np.random.default_rng(3)
    lc = rng.uniform(0.0, 4.0, size=(6, 10))
    lp = rng.uniform(-0.05, 0.2, size=(6, 10))
    m_h = s.f_kn[1] * lc + s.f_p[1] * lp
    m_l = s.f_kn[0] * lc + s.f_p[0] * lp
    w = np.full(lc.shape, 1e4)
    ac, ap = fbp.cdm(s, m_h, m_l, w, w, iters=30)
    # with rho = 0 the fit is exact for a linear forward model (a 2x2 solve per ray), then a >= 0
    assert np.allclose(ac, lc, rtol=1e-8, atol=1e-8)
    assert np.allclose(ap, np.maximum(lp, 0.0), rtol=1e-8, atol=1e-8)
    assert np.all(ap[lp < 0] == 0.0)


def test_cdm_fbp_of_noise_free_polychromatic_data():
    # two overlapping disks with different Compton / PE ratios, Kramers spectra: the decomposition
    # inverts the polychromatic model per ray (beam hardening removed), FBP then images each basis
    g = G.parallel_geometry(64, 180, 128, 0.1, 0.1)
    one = lambda *v: np.array(v, dtype=np.float64)
    ph = P.Phantom(shape=np.array([P.ELLIPSE, P.ELLIPSE]), cx=one(0.0, 0.8), cy=one(0.0, 0.5),
                   a=one(2.5, 0.8), b=one(2.5, 0.8), phi=one(0.0, 0.0), compton=one(0.2, 0.3), pe=one(0.002, 0.03))
    t = spectra.SpectralTables(e_ref_kev=100.0)
    lc, lp = P.line_integrals(ph, g)
    d = P.noise_free_measurements(t, lc, lp)
    m_h, m_l = d["m_h"], d["m_l"]
    w = np.full(lc.shape, 1e5)
    ac, ap = fbp.cdm(t, m_h, m_l, w, w, iters=40)
    assert np.allclose(ac, lc, rtol=1e-6, atol=1e-7) and np.allclose(ap, lp, rtol=1e-5, atol=1e-7)
    xc, xp = fbp.cdm_fbp(g, t, m_h, m_l, w, w, iters=40)
    r0, r1 = _radius_map(g, 0.0, 0.0), _radius_map(g, 0.8, 0.5)
    body = (r0 < 2.0) & (r1 > 1.1)
    insert = r1 < 0.6
    assert abs(xc[body].mean() - 0.2) < 2e-3 and abs(xc[insert].mean() - 0.5) < 5e-3
    assert abs(xp[body].mean() - 0.002) < 1e-4 and abs(xp[insert].mean() - 0.032) < 5e-4


def test_cdm_fbp_start_of_the_admm():
    # the paper's initial image (Sec. 4): CDM-FBP Compton, clamped, and kappa times it for PE
    from oracle import admm

    g = G.parallel_geometry(64, 180, 128, 0.1, 0.1)
    one = lambda *v: np.array(v, dtype=np.float64)
    ph = P.Phantom(shape=np.array([P.ELLIPSE, P.ELLIPSE]), cx=one(0.0, 0.8), cy=one(0.0, 0.5),
                   a=one(2.5, 0.8), b=one(2.5, 0.8), phi=one(0.0, 0.0), compton=one(0.2, 0.3), pe=one(0.002, 0.03))
    t = spectra.SpectralTables(e_ref_kev=100.0)
    lc, lp = P.line_integrals(ph, g)
    d = P.noise_free_measurements(t, lc, lp)
    w = np.full(lc.shape, 1e5)
    prob = admm.Problem(g, t, d["m_h"], d["m_l"], w, w, admm.Params(init=admm.INIT_CDM_FBP, init_udm_iters=40,
                                                                       kappa=0.25))
    xc, xp = admm.initial_image(prob)
    assert prob.count.f == 4 * 40
    assert np.all(xc >= 0) and np.array_equal(xp, 0.25 * xc)
    r0, r1 = _radius_map(g, 0.0, 0.0), _radius_map(g, 0.8, 0.5)
    body, insert = (r0 < 2.0) & (r1 > 1.1), r1 < 0.6
    assert abs(xc[body].mean() - 0.2) < 2e-3 and abs(xc[insert].mean() - 0.5) < 5e-3
