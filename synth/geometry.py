"""Scanner geometry descriptions for the synthetic workloads.

A geometry is plain data: image grid, view angles and detector sampling. The
paper's experiments are 2-D parallel beam (Sec. 4); the fan-beam (flat
detector) variant describes the baggage-like workloads. Conventions:

  * pixel (row j, column i) has its centre at ((i-(nx-1)/2)*pix, (j-(ny-1)/2)*pix) cm;
    images are stored row-major [ny][nx].
  * view v has angle theta_v = angle0 + v*span/n_views.
  * detector bin k sits at u_k = (k-(nb-1)/2)*du + u_offset cm.
  * parallel beam: the ray of (v, k) passes through u_k*(cos, sin)(theta_v) with
    direction (-sin, cos)(theta_v).
  * fan beam, flat detector: source at sod*(cos, sin)(theta_v), detector centre
    at -(sdd-sod)*(cos, sin)(theta_v), detector axis (-sin, cos)(theta_v); the
    ray of bin k runs from the source to the bin centre.

`rays()` gives each ray's origin and unit direction in FP64 for the analytic
line integrals of the phantom module; it is data preparation, not part of the
reconstruction.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PARALLEL = 0
FAN_FLAT = 1


@dataclasses.dataclass(frozen=True)
class Geometry:
    kind: int
    nx: int
    ny: int
    pixel_cm: float
    n_views: int
    angle0_rad: float
    angle_span_rad: float
    n_bins: int
    bin_pitch_cm: float
    bin_offset_cm: float = 0.0
    sod_cm: float = 0.0
    sdd_cm: float = 0.0

    @property
    def n_rays(self) -> int:
        return self.n_views * self.n_bins

    @property
    def n_pixels(self) -> int:
        return self.nx * self.ny

    def angles(self) -> np.ndarray:
        return self.angle0_rad + np.arange(self.n_views, dtype=np.float64) * (self.angle_span_rad / self.n_views)

    def bin_positions(self) -> np.ndarray:
        return (np.arange(self.n_bins, dtype=np.float64) - 0.5 * (self.n_bins - 1)) * self.bin_pitch_cm + self.bin_offset_cm

    def rays(self, views=None):
        """(px, py, dx, dy) arrays of shape [V, Nb]: a point on each ray and its unit direction."""
        th = self.angles() if views is None else self.angles()[np.asarray(views)]
        c = np.cos(th)[:, None]
        s = np.sin(th)[:, None]
        u = self.bin_positions()[None, :]
        if self.kind == PARALLEL:
            px = u * c
            py = u * s
            dx = np.broadcast_to(-s, px.shape).copy()
            dy = np.broadcast_to(c, px.shape).copy()
            return px, py, dx, dy
        if self.kind == FAN_FLAT:
            sx = self.sod_cm * c
            sy = self.sod_cm * s
            qx = -(self.sdd_cm - self.sod_cm) * c - u * s
            qy = -(self.sdd_cm - self.sod_cm) * s + u * c
            ex = qx - sx
            ey = qy - sy
            ln = np.sqrt(ex * ex + ey * ey)
            return np.broadcast_to(sx, ex.shape).copy(), np.broadcast_to(sy, ex.shape).copy(), ex / ln, ey / ln
        raise ValueError(f"unknown geometry kind {self.kind}")

    def as_dict(self) -> dict:
        return dataclasses.asdict(self)


def parallel_geometry(n: int, n_views: int, n_bins: int, pixel_cm: float, bin_pitch_cm: float,
                      span_rad: float = math.pi, angle0_rad: float = 0.0) -> Geometry:
    return Geometry(PARALLEL, n, n, pixel_cm, n_views, angle0_rad, span_rad, n_bins, bin_pitch_cm)


def fan_geometry(n: int, n_views: int, n_bins: int, sod_cm: float = 55.0, sdd_cm: float = 95.0,
                 side_cm: float = 51.2, angle0_rad: float = 0.0) -> Geometry:
    """Fan beam over 2*pi with the detector sized to cover the image's circumscribed circle.

    Reading of the baggage-scanner geometry: the image side is side_cm for every
    N (pixel = side/N), and the flat detector spans 2*sdd*tan(asin(R/sod)) with
    R = side/sqrt(2), split into n_bins bins.
    """
    radius = side_cm / math.sqrt(2.0)
    du = 2.0 * sdd_cm * math.tan(math.asin(radius / sod_cm)) / n_bins
    return Geometry(FAN_FLAT, n, n, side_cm / n, n_views, angle0_rad, 2.0 * math.pi, n_bins, du, 0.0, sod_cm, sdd_cm)


def small_parallel_geometry() -> Geometry:
    """64x64 image of 1 mm pixels, 90 views over 180 degrees, 96 bins of 1 mm."""
    return parallel_geometry(64, 90, 96, 0.1, 0.1)


def baggage_fan_geometry(n: int = 512, n_views: int = 720, n_bins: int = 1024) -> Geometry:
    """Fan beam, source-isocentre 55 cm, source-detector 95 cm, 51.2 cm field."""
    return fan_geometry(n, n_views, n_bins)
