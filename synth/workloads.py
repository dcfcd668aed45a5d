"""Seeded workloads shaped like the paper's scans (Sec. 4).

  * `small_parallel_case`: 64x64 image (1 mm pixels), 90 views over 180 degrees,
    96 bins; a body ellipse with five inserts; Compton in [0, 0.4] cm^-1 and PE
    in [0, 4e-3]; I0 = 1e5.
  * `baggage_fan_case`: fan beam (55 / 95 cm), 512x512, 720 views over 360
    degrees, 1024 bins; 40 ellipses/rectangles, 10% of them high-Z inserts
    (Compton 1-2 cm^-1, PE 0.1-0.5); I0 = 2e5.
Every case is a dict with the geometry, spectral tables, phantom, truth images
and the Poisson data (FP64), all drawn from numpy PCG64 with seed = base + slice.
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import Geometry, baggage_fan_geometry, fan_geometry, small_parallel_geometry
from .phantom import ELLIPSE, RECTANGLE, Phantom, SupersampledMaps, line_integrals, measurements
from .spectra import SpectralTables

BASE_SEED = 1905


def _draw_objects(rng, n, sample_one, maps: SupersampledMaps, c_max, p_max, max_tries=200):
    rows = []
    for _ in range(n):
        for _try in range(max_tries):
            row = sample_one(rng, len(rows))
            ph = _phantom_from_rows([row])
            sub = maps.paint(ph, 0)
            if sub is None:
                continue
            bc = maps.xc[sub]
            bp = maps.xp[sub]
            if bc.min() < -1e-12 or bp.min() < -1e-12 or bc.max() > c_max + 1e-12 or bp.max() > p_max + 1e-12:
                maps.paint(ph, 0, -1.0)
                continue
            rows.append(row)
            break
        else:
            raise RuntimeError("phantom sampler could not place an object inside the value range")
    return _phantom_from_rows(rows)


def _phantom_from_rows(rows) -> Phantom:
    arr = np.array(rows, dtype=np.float64).reshape(-1, 8)
    return Phantom(arr[:, 0].astype(np.int64), arr[:, 1], arr[:, 2], arr[:, 3], arr[:, 4], arr[:, 5],
                   arr[:, 6], arr[:, 7])


def small_phantom(geom: Geometry, rng, c_max=0.4, p_max=4e-3, supersample=4):
    half = 0.5 * geom.nx * geom.pixel_cm

    def sample(rng, idx):
        if idx == 0:
            a = rng.uniform(0.8, 0.9) * half
            b = rng.uniform(0.8, 0.9) * half
            return [ELLIPSE, 0.0, 0.0, a, b, rng.uniform(0, math.pi), 0.5 * c_max, 0.5 * p_max]
        r = 0.6 * half * math.sqrt(rng.uniform())
        t = rng.uniform(0, 2 * math.pi)
        return [ELLIPSE, r * math.cos(t), r * math.sin(t), rng.uniform(0.05, 0.3) * half,
                rng.uniform(0.05, 0.3) * half, rng.uniform(0, math.pi),
                rng.uniform(-0.5, 0.5) * c_max, rng.uniform(-0.5, 0.5) * p_max]

    maps = SupersampledMaps(geom, supersample)
    ph = _draw_objects(rng, 6, sample, maps, c_max, p_max)
    return ph, maps.pixel_average()


def baggage_phantom(geom: Geometry, rng, n_objects=40, c_max=2.0, p_max=0.5, supersample=4):
    half = 0.5 * geom.nx * geom.pixel_cm

    def sample(rng, idx):
        shape = ELLIPSE if rng.uniform() < 0.5 else RECTANGLE
        high_z = rng.uniform() < 0.1
        if high_z:
            a, b = rng.uniform(0.01, 0.05, size=2) * half
            c, p = rng.uniform(1.0, 2.0), rng.uniform(0.1, 0.5)
        else:
            a, b = rng.uniform(0.03, 0.25, size=2) * half
            c, p = rng.uniform(0.1, 0.4), rng.uniform(0.0, 4e-3)
        r = 0.75 * half * math.sqrt(rng.uniform())
        t = rng.uniform(0, 2 * math.pi)
        return [shape, r * math.cos(t), r * math.sin(t), a, b, rng.uniform(0, math.pi), c, p]

    maps = SupersampledMaps(geom, supersample)
    ph = _draw_objects(rng, n_objects, sample, maps, c_max, p_max)
    return ph, maps.pixel_average()


def make_case(geom: Geometry, phantom_fn, i0: float, seed: int, e_ref_kev: float = 1.0, noise: bool = True):
    rng = np.random.Generator(np.random.PCG64(seed))
    ph, (xc, xp) = phantom_fn(geom, rng)
    spec = SpectralTables(e_ref_kev=e_ref_kev)
    lc, lp = line_integrals(ph, geom)
    if noise:
        data = measurements(spec, lc, lp, i0, seed + 1_000_000)
    else:
        from .phantom import noise_free_measurements
        data = noise_free_measurements(spec, lc, lp)
    return {"geom": geom, "spectra": spec, "phantom": ph, "truth_c": xc, "truth_p": xp,
            "L_c": lc, "L_p": lp, "i0": i0, "seed": seed, **data}


def small_parallel_case(slice_index: int = 0, e_ref_kev: float = 1.0, noise: bool = True):
    return make_case(small_parallel_geometry(), small_phantom, 1e5, BASE_SEED + slice_index, e_ref_kev, noise)


def baggage_fan_case(slice_index: int = 0, n: int = 512, n_views: int = 720, n_bins: int = 1024,
                     e_ref_kev: float = 100.0, noise: bool = True):
    geom = baggage_fan_geometry(n, n_views, n_bins) if (n, n_views, n_bins) == (512, 720, 1024) else fan_geometry(n, n_views, n_bins)
    return make_case(geom, baggage_phantom, 2e5, BASE_SEED + slice_index, e_ref_kev, noise)


# Reading for the baggage workloads: their photoelectric range (up to 0.5) is physical with the E^-3
# basis referred to 100 keV; the initial PE image is kappa = PE max / Compton max = 0.25 times Compton.
BAGGAGE_E_REF_KEV = 100.0
BAGGAGE_KAPPA = 0.25
SMALL_KAPPA = 1e-2
# seed base of the mixed-precision workload's slices (1024 x 1024, 1440 views, 2048 bins)
MIXED_SEED_BASE = 5000

# --- ADMM parameters of the paper's experiments (Sec. 4): lambda = 1e-5, rho0 = 1e-3 for both bases.
PAPER_LAMBDA = 1e-5
PAPER_RHO0 = 1e-3


def uneven_batch_shapes(n_slices: int = 64, seed: int = BASE_SEED):
    """Seeded (N, views, bins) of the batched uneven-slice workload: N in 256..1024 step 64,
    views in 360..1440 step 90, bins in 512..2048 step 128."""
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    n = rng.integers(0, (1024 - 256) // 64 + 1, n_slices) * 64 + 256
    v = rng.integers(0, (1440 - 360) // 90 + 1, n_slices) * 90 + 360
    b = rng.integers(0, (2048 - 512) // 128 + 1, n_slices) * 128 + 512
    return [(int(a), int(c), int(d)) for a, c, d in zip(n, v, b)]


def quick_fan_case(slice_index: int, n: int, n_views: int, n_bins: int, n_objects: int = 12,
                   e_ref_kev: float = BAGGAGE_E_REF_KEV, i0: float = 2e5):
    """A fan-beam slice with a light phantom and no truth image (for large batched runs)."""
    geom = fan_geometry(n, n_views, n_bins)
    seed = BASE_SEED + 10_000 + slice_index
    rng = np.random.Generator(np.random.PCG64(seed))
    half = 0.5 * geom.nx * geom.pixel_cm
    rows = []
    for k in range(n_objects):
        shape = ELLIPSE if rng.uniform() < 0.5 else RECTANGLE
        high_z = k == 0
        a, b = (rng.uniform(0.02, 0.05, 2) if high_z else rng.uniform(0.05, 0.25, 2)) * half
        c, p = (rng.uniform(1.0, 2.0), rng.uniform(0.1, 0.5)) if high_z else (rng.uniform(0.1, 0.3), rng.uniform(0, 4e-3))
        r = 0.7 * half * math.sqrt(rng.uniform())
        t = rng.uniform(0, 2 * math.pi)
        rows.append([shape, r * math.cos(t), r * math.sin(t), a, b, rng.uniform(0, math.pi), c, p])
    ph = _phantom_from_rows(rows)
    spec = SpectralTables(e_ref_kev=e_ref_kev)
    lc, lp = line_integrals(ph, geom)
    data = measurements(spec, lc, lp, i0, seed + 1_000_000)
    return {"geom": geom, "spectra": spec, "phantom": ph, "i0": i0, "seed": seed, **data}
