"""Seeded ellipse/rectangle phantoms, their analytic line integrals and Poisson data.

The paper's phantoms (sim18, Water, Clutter; Sec. 4) are not available, so the
workloads use synthetic phantoms of the same sizes. Each object is an ellipse or
a rotated rectangle with additive Compton and photoelectric coefficients.

  * `truth_image` rasterises the phantom by supersampled pixel averaging; it is
    the ground truth x* of the quality metric (Eq. 14).
  * `line_integrals` is the exact (continuous) Radon transform: closed-form
    chord lengths of each ray through each object, so the data are not made
    with any discrete projector (no inverse crime).
  * `measurements` draws photon counts N ~ Poisson(I0 * sum_E S(E) exp(-f_KN(E) L_c - f_p(E) L_p))
    (the measurement model of Eq. 2 with the integral over E as a sum over
    unit-sum spectral bins) and returns m = -ln(max(N,1)/I0) and the weights
    w = max(N,1) (photon counts on the diagonal of Sigma, Eq. 4).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .geometry import Geometry
from .spectra import SpectralTables

ELLIPSE = 0
RECTANGLE = 1


@dataclasses.dataclass
class Phantom:
    # one row per object: shape, cx, cy, semi-axis a, semi-axis b, angle phi, compton, pe
    shape: np.ndarray
    cx: np.ndarray
    cy: np.ndarray
    a: np.ndarray
    b: np.ndarray
    phi: np.ndarray
    compton: np.ndarray
    pe: np.ndarray

    @property
    def n_objects(self) -> int:
        return int(self.shape.size)


def _inside(ph: Phantom, idx: int, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    c, s = np.cos(ph.phi[idx]), np.sin(ph.phi[idx])
    dx = x - ph.cx[idx]
    dy = y - ph.cy[idx]
    qx = c * dx + s * dy
    qy = -s * dx + c * dy
    if ph.shape[idx] == ELLIPSE:
        return (qx / ph.a[idx]) ** 2 + (qy / ph.b[idx]) ** 2 <= 1.0
    return (np.abs(qx) <= ph.a[idx]) & (np.abs(qy) <= ph.b[idx])


class SupersampledMaps:
    """Compton/PE maps on a grid of supersample^2 points per pixel (for painting and checks)."""

    def __init__(self, geom: Geometry, supersample: int = 4):
        ss = supersample
        off = (np.arange(ss) + 0.5) / ss - 0.5
        self.geom = geom
        self.ss = ss
        self.xs = ((np.arange(geom.nx) - 0.5 * (geom.nx - 1))[:, None] + off[None, :]).ravel() * geom.pixel_cm
        self.ys = ((np.arange(geom.ny) - 0.5 * (geom.ny - 1))[:, None] + off[None, :]).ravel() * geom.pixel_cm
        self.xc = np.zeros((self.ys.size, self.xs.size))
        self.xp = np.zeros_like(self.xc)

    def paint(self, ph: Phantom, o: int, sign: float = 1.0):
        """Add (sign=+1) or remove (sign=-1) object o; returns the touched index block."""
        r = max(ph.a[o], ph.b[o]) * 1.4143
        ci = np.nonzero(np.abs(self.xs - ph.cx[o]) <= r)[0]
        cj = np.nonzero(np.abs(self.ys - ph.cy[o]) <= r)[0]
        if ci.size == 0 or cj.size == 0:
            return None
        X, Y = np.meshgrid(self.xs[ci], self.ys[cj])
        m = _inside(ph, o, X, Y)
        sub = np.ix_(cj, ci)
        self.xc[sub] += sign * m * ph.compton[o]
        self.xp[sub] += sign * m * ph.pe[o]
        return sub

    def pixel_average(self):
        g, ss = self.geom, self.ss
        return (self.xc.reshape(g.ny, ss, g.nx, ss).mean(axis=(1, 3)),
                self.xp.reshape(g.ny, ss, g.nx, ss).mean(axis=(1, 3)))


def truth_image(ph: Phantom, geom: Geometry, supersample: int = 4):
    """(x_c, x_p): [ny][nx] FP64 pixel averages over supersample^2 points per pixel."""
    maps = SupersampledMaps(geom, supersample)
    for o in range(ph.n_objects):
        maps.paint(ph, o)
    return maps.pixel_average()


def chord_lengths(ph: Phantom, idx: int, px, py, dx, dy) -> np.ndarray:
    """Length of each ray (point p, unit direction d) inside object idx, in cm."""
    c, s = np.cos(ph.phi[idx]), np.sin(ph.phi[idx])
    ox = px - ph.cx[idx]
    oy = py - ph.cy[idx]
    qx = c * ox + s * oy
    qy = -s * ox + c * oy
    ex = c * dx + s * dy
    ey = -s * dx + c * dy
    a, b = ph.a[idx], ph.b[idx]
    if ph.shape[idx] == ELLIPSE:
        A = (ex / a) ** 2 + (ey / b) ** 2
        B = 2.0 * (qx * ex / a**2 + qy * ey / b**2)
        C = (qx / a) ** 2 + (qy / b) ** 2 - 1.0
        disc = B * B - 4.0 * A * C
        return np.where(disc > 0.0, np.sqrt(np.maximum(disc, 0.0)) / A, 0.0)
    # rectangle: intersect the two slabs |q + t e| <= half-width
    with np.errstate(divide="ignore", invalid="ignore"):
        t_lo = np.full(qx.shape, -np.inf)
        t_hi = np.full(qx.shape, np.inf)
        for q, e, h in ((qx, ex, a), (qy, ey, b)):
            par = np.abs(e) < 1e-300
            t1 = (-h - q) / e
            t2 = (h - q) / e
            lo = np.where(par, np.where(np.abs(q) <= h, -np.inf, np.inf), np.minimum(t1, t2))
            hi = np.where(par, np.where(np.abs(q) <= h, np.inf, -np.inf), np.maximum(t1, t2))
            t_lo = np.maximum(t_lo, lo)
            t_hi = np.minimum(t_hi, hi)
    return np.maximum(t_hi - t_lo, 0.0)


def line_integrals(ph: Phantom, geom: Geometry, views=None):
    """(L_c, L_p): [V][Nb] FP64 exact line integrals of the Compton and PE maps."""
    px, py, dx, dy = geom.rays(views)
    lc = np.zeros(px.shape)
    lp = np.zeros(px.shape)
    for o in range(ph.n_objects):
        L = chord_lengths(ph, o, px, py, dx, dy)
        lc += ph.compton[o] * L
        lp += ph.pe[o] * L
    return lc, lp


def expected_transmission(spec: SpectralTables, lc: np.ndarray, lp: np.ndarray, chunk: int = 1 << 16):
    """(t_h, t_l) = sum_E S(E) exp(-f_KN(E) L_c - f_p(E) L_p) per ray (unit-sum spectra)."""
    lc = np.asarray(lc, dtype=np.float64).ravel()
    lp = np.asarray(lp, dtype=np.float64).ravel()
    th = np.empty_like(lc)
    tl = np.empty_like(lc)
    for s0 in range(0, lc.size, chunk):
        sl = slice(s0, s0 + chunk)
        att = np.exp(-np.outer(lc[sl], spec.f_kn) - np.outer(lp[sl], spec.f_p))
        th[sl] = att @ spec.s_high
        tl[sl] = att @ spec.s_low
    return th, tl


def measurements(spec: SpectralTables, lc: np.ndarray, lp: np.ndarray, i0: float, seed: int):
    """Poisson data: dict of m_h, m_l, w_h, w_l shaped like lc (FP64)."""
    shape = np.shape(lc)
    th, tl = expected_transmission(spec, lc, lp)
    rng = np.random.Generator(np.random.PCG64(seed))
    nh = rng.poisson(i0 * th).astype(np.float64)
    nl = rng.poisson(i0 * tl).astype(np.float64)
    nh = np.maximum(nh, 1.0)
    nl = np.maximum(nl, 1.0)
    return {
        "m_h": (-np.log(nh / i0)).reshape(shape),
        "m_l": (-np.log(nl / i0)).reshape(shape),
        "w_h": nh.reshape(shape),
        "w_l": nl.reshape(shape),
    }


def noise_free_measurements(spec: SpectralTables, lc: np.ndarray, lp: np.ndarray):
    """m = -ln(t) without noise, unit weights (for recovery tests)."""
    shape = np.shape(lc)
    th, tl = expected_transmission(spec, lc, lp)
    return {
        "m_h": (-np.log(th)).reshape(shape),
        "m_l": (-np.log(tl)).reshape(shape),
        "w_h": np.ones(shape),
        "w_l": np.ones(shape),
    }
