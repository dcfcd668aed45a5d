"""Build and load the oracle's C part (oracle_dect.c) with gcc; FP64, no fast-math.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_dect.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_dect.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's shared library (OpenMP if available) and return its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OGGeom(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nv", ctypes.c_int),
                ("nb", ctypes.c_int), ("pix", ctypes.c_double), ("ang0", ctypes.c_double),
                ("span", ctypes.c_double), ("du", ctypes.c_double), ("uoff", ctypes.c_double),
                ("sod", ctypes.c_double), ("sdd", ctypes.c_double)]


def geom_struct(g) -> OGGeom:
    return OGGeom(g.kind, g.nx, g.ny, g.n_views, g.n_bins, g.pixel_cm, g.angle0_rad, g.angle_span_rad,
                  g.bin_pitch_cm, g.bin_offset_cm, g.sod_cm, g.sdd_cm)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            gp = ctypes.POINTER(OGGeom)
            L.og_num_threads.restype = ctypes.c_int
            L.og_project.argtypes = [gp, dp, dp]
            L.og_backproject.argtypes = [gp, dp, dp]
            L.og_project_ray.argtypes = [gp, dp, ctypes.c_int, ctypes.c_int]
            L.og_project_ray.restype = ctypes.c_double
            L.og_ray_weights.argtypes = [gp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), dp, ctypes.c_int]
            L.og_ray_weights.restype = ctypes.c_int
            L.og_forward_model.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_long, dp, dp, dp, dp, dp]
            L.og_udm.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_long, dp, dp, dp, dp, dp, dp,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp, dp,
                                 ctypes.POINTER(ctypes.c_uint8)]
            L.og_udm_cost.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_long, dp, dp, dp, dp, dp, dp,
                                      ctypes.c_double, ctypes.c_double, dp, dp, dp]
            _lib = L
    return _lib


def dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return int(lib().og_num_threads())
