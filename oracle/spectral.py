"""Spectral forward model f (Eq. 3) and the per-ray decomposition UDM (Eq. 13), FP64.

TEST INFRASTRUCTURE ONLY. The arithmetic is in oracle_dect.c; these wrappers
marshal numpy arrays. Spectra are normalised to unit sum inside, so the
constants C_{h/l} of Eq. 3 vanish (f(0) = 0).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _clib


def _tables(spec):
    t = [np.ascontiguousarray(getattr(spec, n), dtype=np.float64) for n in ("s_high", "s_low", "f_kn", "f_p")]
    return t


def forward_model(spec, a_c, a_p, jacobian: bool = False):
    """f_h, f_l (and the 4 Jacobian entries df_h/da_c, df_h/da_p, df_l/da_c, df_l/da_p) per ray."""
    a_c = np.ascontiguousarray(a_c, dtype=np.float64).ravel()
    a_p = np.ascontiguousarray(a_p, dtype=np.float64).ravel()
    n = a_c.size
    fh = np.empty(n)
    fl = np.empty(n)
    jac = np.empty((n, 4)) if jacobian else None
    sh, sl, fkn, fp = _tables(spec)
    _clib.lib().og_forward_model(fkn.size, _clib.dptr(sh), _clib.dptr(sl), _clib.dptr(fkn), _clib.dptr(fp),
                                 n, _clib.dptr(a_c), _clib.dptr(a_p), _clib.dptr(fh), _clib.dptr(fl),
                                 _clib.dptr(jac) if jacobian else None)
    return (fh, fl, jac) if jacobian else (fh, fl)


def udm(spec, m_h, m_l, w_h, w_l, v_c, v_p, rho_c: float, rho_p: float, iters: int, a_c, a_p, mu):
    """Eq. 13 by LM for every ray; returns new (a_c, a_p, mu, status). Inputs are not modified."""
    arrs = [np.ascontiguousarray(x, dtype=np.float64).ravel() for x in (m_h, m_l, w_h, w_l, v_c, v_p)]
    ac = np.array(a_c, dtype=np.float64).ravel()
    ap = np.array(a_p, dtype=np.float64).ravel()
    mu_ = np.array(mu, dtype=np.float64).ravel()
    n = ac.size
    st = np.zeros(n, dtype=np.uint8)
    sh, sl, fkn, fp = _tables(spec)
    _clib.lib().og_udm(fkn.size, _clib.dptr(sh), _clib.dptr(sl), _clib.dptr(fkn), _clib.dptr(fp), n,
                       *[_clib.dptr(x) for x in arrs], float(rho_c), float(rho_p), int(iters),
                       _clib.dptr(ac), _clib.dptr(ap), _clib.dptr(mu_),
                       st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return ac, ap, mu_, st


def udm_cost(spec, m_h, m_l, w_h, w_l, v_c, v_p, rho_c: float, rho_p: float, a_c, a_p):
    """Eq. 13's per-ray cost at (a_c, a_p)."""
    arrs = [np.ascontiguousarray(x, dtype=np.float64).ravel() for x in (m_h, m_l, w_h, w_l, v_c, v_p, a_c, a_p)]
    n = arrs[0].size
    out = np.empty(n)
    sh, sl, fkn, fp = _tables(spec)
    _clib.lib().og_udm_cost(fkn.size, _clib.dptr(sh), _clib.dptr(sl), _clib.dptr(fkn), _clib.dptr(fp), n,
                            *[_clib.dptr(x) for x in arrs[:6]], float(rho_c), float(rho_p),
                            _clib.dptr(arrs[6]), _clib.dptr(arrs[7]), _clib.dptr(out))
    return out
