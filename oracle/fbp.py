"""Filtered backprojection and the CDM-FBP comparison method (Sec. 2, Sec. 4), FP64.

TEST INFRASTRUCTURE ONLY: plain numpy, one view at a time.

The paper's baseline (i) decomposes each ray's dual-energy measurements into Compton and PE line
integrals (the constrained decomposition method, CDM, from a cited reference) and then
reconstructs each basis by filtered backprojection (FBP); its Compton image also starts the ADMM.
The paper restates neither, so both follow these readings:

  * CDM: Eq. 13 with rho_c = rho_p = 0, i.e. the weighted least-squares fit of the forward model
    f(a) to (m_h, m_l) per ray, by `iters` Levenberg-Marquardt iterations (the same LM as UDM)
    from a_c = m_l / sum_E S_l f_KN, a_p = 0; then the constraint a_beta >= 0 per basis (line
    integrals of non-negative attenuation), applied to the result.
  * FBP: the textbook algorithm with the band-limited ramp filter, on the geometry of the
    projector (bin u_k = (k - (Nb-1)/2) du + u_offset):
      - ramp kernel on a sampling of pitch alpha: h(0) = 1/(4 alpha^2), h(m alpha) = 0 for even
        m != 0, -1/(m^2 pi^2 alpha^2) for odd m; filtered row Q(n) = alpha sum_k h((n-k) alpha) p(k)
        (its frequency response is the ramp |nu| up to the Nyquist frequency);
      - parallel beam over pi or 2 pi: x(P) = (pi / V) sum_v Q_v(t), t = P . (cos, sin)(theta_v);
      - flat-detector fan beam over 2 pi: the detector rescaled to the isocentre, s = u SOD/SDD,
        alpha = du SOD/SDD; pre-weight SOD / sqrt(SOD^2 + s^2); half the ramp; x(P) =
        (2 pi / V) sum_v Q_v(s(P)) / U^2 with U = (SOD - P . n_v) / SOD and s(P) = (P . e_v) / U,
        n_v = (cos, sin)(beta_v) towards the source and e_v = (-sin, cos)(beta_v) the detector axis;
      - Q between bins by linear interpolation, zero beyond the first and last bin.
    Other angular spans (short scans) are not supported.
"""
from __future__ import annotations

import numpy as np

from . import spectral


def ramp_kernel(n_bins: int, alpha: float) -> np.ndarray:
    """h(m alpha) for m = -(n_bins - 1) .. n_bins - 1 (index m + n_bins - 1)."""
    m = np.arange(-(n_bins - 1), n_bins)
    h = np.zeros(m.shape)
    h[m == 0] = 1.0 / (4.0 * alpha * alpha)
    odd = (m % 2) != 0
    h[odd] = -1.0 / (m[odd].astype(np.float64) ** 2 * np.pi**2 * alpha * alpha)
    return h


def filter_rows(p: np.ndarray, alpha: float) -> np.ndarray:
    """Q[v][n] = alpha sum_k h((n - k) alpha) p[v][k] (linear convolution, no wrap-around)."""
    V, nb = p.shape
    h = ramp_kernel(nb, alpha)
    idx = np.arange(nb)
    T = h[(idx[:, None] - idx[None, :]) + nb - 1]   # T[n][k] = h(n - k)
    return alpha * (p @ T.T)


def _interp(q: np.ndarray, kf: np.ndarray) -> np.ndarray:
    """Linear interpolation of one filtered row at fractional bins kf, zero beyond bins 0 .. nb-1."""
    nb = q.shape[0]
    qp = np.concatenate([[0.0], q, [0.0]])          # qp[k + 1] = q[k], zero at k = -1 and k = nb
    k0 = np.floor(kf)
    f = kf - k0
    inside = (k0 >= -1) & (k0 <= nb - 1)
    i0 = np.clip(k0, -1, nb - 1).astype(np.int64) + 1
    v = (1.0 - f) * qp[i0] + f * qp[np.minimum(i0 + 1, nb + 1)]
    return np.where(inside, v, 0.0)


def fbp(geom, sino: np.ndarray) -> np.ndarray:
    """Filtered backprojection of one sinogram [V][Nb] to an image [ny][nx]."""
    g = geom
    p = np.asarray(sino, dtype=np.float64).reshape(g.n_views, g.n_bins)
    th = g.angles()
    u = g.bin_positions()
    ii, jj = np.meshgrid(np.arange(g.nx), np.arange(g.ny))
    X = (ii - 0.5 * (g.nx - 1)) * g.pixel_cm
    Y = (jj - 0.5 * (g.ny - 1)) * g.pixel_cm
    x = np.zeros((g.ny, g.nx))
    if g.kind == 0:
        if not (np.isclose(g.angle_span_rad, np.pi) or np.isclose(g.angle_span_rad, 2 * np.pi)):
            raise ValueError("parallel-beam FBP needs views over pi or 2 pi")
        Q = filter_rows(p, g.bin_pitch_cm)
        for v in range(g.n_views):
            t = X * np.cos(th[v]) + Y * np.sin(th[v])
            kf = (t - g.bin_offset_cm) / g.bin_pitch_cm + 0.5 * (g.n_bins - 1)
            x += _interp(Q[v], kf)
        return x * (np.pi / g.n_views)
    if g.kind == 1:
        if not np.isclose(g.angle_span_rad, 2 * np.pi):
            raise ValueError("fan-beam FBP needs views over 2 pi")
        sod, sdd = g.sod_cm, g.sdd_cm
        s = u * (sod / sdd)
        alpha = g.bin_pitch_cm * (sod / sdd)
        Q = 0.5 * filter_rows(p * (sod / np.sqrt(sod * sod + s * s))[None, :], alpha)
        for v in range(g.n_views):
            c, sn = np.cos(th[v]), np.sin(th[v])
            U = (sod - (X * c + Y * sn)) / sod
            sp = (-X * sn + Y * c) / U
            kf = (sp * (sdd / sod) - g.bin_offset_cm) / g.bin_pitch_cm + 0.5 * (g.n_bins - 1)
            x += _interp(Q[v], kf) / (U * U)
        return x * (2.0 * np.pi / g.n_views)
    raise ValueError(f"unknown geometry kind {g.kind}")


def cdm_fit(spec, m_h, m_l, w_h, w_l, iters: int = 20, mu0: float = 1e-3):
    """(a_c, a_p) [V][Nb]: the per-ray decomposition with rho = 0, before the constraint."""
    m_h = np.asarray(m_h, dtype=np.float64)
    shape = m_h.shape
    m_l = np.asarray(m_l, dtype=np.float64).reshape(shape)
    sl = spec.s_low / spec.s_low.sum()
    a_c0 = m_l / float(np.dot(sl, spec.f_kn))
    zeros = np.zeros(shape)
    mu = np.full(shape, mu0)
    ac, ap, _, _ = spectral.udm(spec, m_h, m_l, np.asarray(w_h, np.float64).reshape(shape),
                                np.asarray(w_l, np.float64).reshape(shape), zeros, zeros, 0.0, 0.0, iters,
                                a_c0, zeros, mu)
    return ac.reshape(shape), ap.reshape(shape)


def cdm(spec, m_h, m_l, w_h, w_l, iters: int = 20, mu0: float = 1e-3):
    """(a_c, a_p) [V][Nb]: per-ray decomposition with rho = 0, then a >= 0."""
    ac, ap = cdm_fit(spec, m_h, m_l, w_h, w_l, iters, mu0)
    return np.maximum(ac, 0.0), np.maximum(ap, 0.0)


def cdm_fbp(geom, spec, m_h, m_l, w_h, w_l, iters: int = 20):
    """(x_c, x_p): FBP of the CDM line integrals of each basis."""
    ac, ap = cdm(spec, m_h, m_l, w_h, w_l, iters)
    return fbp(geom, ac), fbp(geom, ap)
