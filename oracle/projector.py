"""Forward projector R and its transpose R^T (FP64 oracle).

TEST INFRASTRUCTURE ONLY. R is the projection matrix of Eq. 2 / Eq. 3
(Joseph's ray-driven interpolation, see oracle_dect.c); R^T scatters the same
weights. Images are [ny][nx], sinograms [n_views][n_bins].
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _clib


def project(geom, img: np.ndarray) -> np.ndarray:
    """R x for one image (Eq. 3's R)."""
    img = np.ascontiguousarray(img, dtype=np.float64).reshape(geom.ny, geom.nx)
    out = np.empty((geom.n_views, geom.n_bins))
    g = _clib.geom_struct(geom)
    _clib.lib().og_project(ctypes.byref(g), _clib.dptr(img), _clib.dptr(out))
    return out


def backproject(geom, sino: np.ndarray) -> np.ndarray:
    """R^T y for one sinogram."""
    sino = np.ascontiguousarray(sino, dtype=np.float64).reshape(geom.n_views, geom.n_bins)
    out = np.empty((geom.ny, geom.nx))
    g = _clib.geom_struct(geom)
    _clib.lib().og_backproject(ctypes.byref(g), _clib.dptr(sino), _clib.dptr(out))
    return out


def project_ray(geom, img: np.ndarray, v: int, k: int) -> float:
    img = np.ascontiguousarray(img, dtype=np.float64).reshape(geom.ny, geom.nx)
    g = _clib.geom_struct(geom)
    return float(_clib.lib().og_project_ray(ctypes.byref(g), _clib.dptr(img), int(v), int(k)))


def ray_weights(geom, v: int, k: int):
    """The non-zero entries of row (v, k) of R: (flat pixel indices, weights)."""
    cap = 4 * (geom.nx + geom.ny) + 8
    idx = np.empty(cap, dtype=np.int64)
    w = np.empty(cap)
    g = _clib.geom_struct(geom)
    n = _clib.lib().og_ray_weights(ctypes.byref(g), int(v), int(k),
                                   idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _clib.dptr(w), cap)
    assert n <= cap
    return idx[:n].copy(), w[:n].copy()


def matrix(geom) -> np.ndarray:
    """Dense R (n_rays x n_pixels); only for tiny geometries."""
    R = np.zeros((geom.n_rays, geom.n_pixels))
    for v in range(geom.n_views):
        for k in range(geom.n_bins):
            idx, w = ray_weights(geom, v, k)
            R[v * geom.n_bins + k, idx] = w
    return R
