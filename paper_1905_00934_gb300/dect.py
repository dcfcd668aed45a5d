"""Thin Python binding of the dect C ABI (include/dect.h): argument marshalling only.

Every function forwards to the CUDA library libdect.so built in-tree by
`paper_1905_00934_gb300.build`. There is no CPU fallback: if the library is
missing or no CUDA device is present, the calls raise.

Tensors are torch tensors; device buffers are passed by data pointer and the
call is enqueued on the current torch CUDA stream unless a stream is given.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdect.so")

OK, EINVAL, ENOMEM, ECUDA, EUNSUPPORTED, ETIMEOUT, ENOTCONV = range(7)
PARALLEL, FAN_FLAT = 0, 1
F32, F64 = 0, 1
STORE_F32, STORE_F16, STORE_BF16, STORE_F64 = 0, 1, 2, 3
SCHEME_UDM_PCG, SCHEME_LM_CG = 0, 1
PRECOND_NONE, PRECOND_CIRCULANT, PRECOND_RAMP = 0, 1, 2
INIT_PCG, INIT_CDM_FBP = 0, 1
RAY_ACCEPTED, RAY_REJECTED, RAY_NONFINITE = 0, 1, 2
# dect_admm_get array selectors
X, RX, A, UA, Y, UY, Z, UZ, MU, H = range(10)


class DectError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"dect status {status}: {msg}")
        self.status = status


class GeomDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("n_views", ctypes.c_int32), ("n_bins", ctypes.c_int32), ("pixel_cm", ctypes.c_double),
                ("angle0_rad", ctypes.c_double), ("angle_span_rad", ctypes.c_double),
                ("bin_pitch_cm", ctypes.c_double), ("bin_offset_cm", ctypes.c_double),
                ("sod_cm", ctypes.c_double), ("sdd_cm", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("lambda_c", ctypes.c_double), ("lambda_p", ctypes.c_double), ("rho0_c", ctypes.c_double),
                ("rho0_p", ctypes.c_double), ("m_udm", ctypes.c_int32), ("n_pcg", ctypes.c_int32),
                ("rho_mu", ctypes.c_double), ("rho_tau", ctypes.c_double), ("lm_mu0", ctypes.c_double),
                ("kappa", ctypes.c_double), ("init_udm_iters", ctypes.c_int32), ("init_pcg_iters", ctypes.c_int32),
                ("precondition", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("bp_view_groups", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("scheme", ctypes.c_int32), ("init", ctypes.c_int32),
                ("udm_f64", ctypes.c_int32), ("objective_every", ctypes.c_int32), ("bp_tile", ctypes.c_int32),
                ("bp_cluster", ctypes.c_int32), ("bp_slices", ctypes.c_int32), ("bp_reduce", ctypes.c_int32),
                ("proj_views", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("iteration", ctypes.c_int32), ("rho", ctypes.c_double * 2), ("r_pri", ctypes.c_double * 2),
                ("r_dual", ctypes.c_double * 2), ("xi_db", ctypes.c_double * 2), ("count_R", ctypes.c_int64),
                ("count_RT", ctypes.c_int64), ("count_f", ctypes.c_int64), ("count_launches", ctypes.c_int64),
                ("bp_view_groups", ctypes.c_int32), ("objective", ctypes.c_double),
                ("objective_iteration", ctypes.c_int32), ("bp_tile", ctypes.c_int32), ("bp_cluster", ctypes.c_int32),
                ("bp_slices", ctypes.c_int32), ("bp_reduce", ctypes.c_int32),
                ("proj_views", ctypes.c_int32)]


# every symbol declared in include/dect.h, with its ctypes signature
_VP = ctypes.c_void_p
_SIGS = {
    "dect_version": ([], ctypes.c_char_p),
    "dect_last_error": ([], ctypes.c_char_p),
    "dect_sync": ([_VP], ctypes.c_int),
    "dect_geometry_create": ([ctypes.POINTER(GeomDesc), ctypes.POINTER(_VP)], ctypes.c_int),
    "dect_geometry_destroy": ([_VP], None),
    "dect_spectra_create": ([ctypes.c_int32, _VP, _VP, _VP, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "dect_spectra_destroy": ([_VP], None),
    "dect_project": ([_VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP], ctypes.c_int),
    "dect_backproject": ([_VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP], ctypes.c_int),
    "dect_project_noalloc": ([_VP, ctypes.c_int32, _VP, _VP, _VP], ctypes.c_int),
    "dect_decompose_rays": ([_VP, ctypes.c_int64, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double,
                             ctypes.c_int32, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "dect_fbp": ([_VP, ctypes.c_int32, _VP, _VP, ctypes.c_int32, _VP], ctypes.c_int),
    "dect_cdm_fbp": ([_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int32, _VP, _VP, _VP], ctypes.c_int),
    "dect_forward_model": ([_VP, ctypes.c_int64, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "dect_forward_model_vjp": ([_VP, ctypes.c_int64, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "dect_params_default": ([ctypes.POINTER(Params)], None),
    "dect_admm_create": ([_VP, ctypes.c_int32, _VP, ctypes.POINTER(Params), ctypes.POINTER(_VP)], ctypes.c_int),
    "dect_admm_destroy": ([_VP], None),
    "dect_admm_set_data": ([_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "dect_admm_set_truth": ([_VP, ctypes.c_int32, _VP, _VP], ctypes.c_int),
    "dect_admm_step": ([_VP, ctypes.c_int32, _VP], ctypes.c_int),
    "dect_reconstruct": ([_VP, ctypes.c_int32, _VP], ctypes.c_int),
    "dect_admm_get": ([_VP, ctypes.c_int32, ctypes.c_int32, _VP, ctypes.c_size_t, _VP], ctypes.c_int),
    "dect_admm_stats": ([_VP, ctypes.c_int32, ctypes.POINTER(Stats), _VP], ctypes.c_int),
    "dect_admm_profile": ([_VP, ctypes.c_int32, _VP, _VP, _VP], ctypes.c_int),
    "dect_admm_state_bytes": ([_VP, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "dect_admm_save": ([_VP, _VP, ctypes.c_size_t, _VP], ctypes.c_int),
    "dect_admm_load": ([_VP, _VP, ctypes.c_size_t, _VP], ctypes.c_int),
}

_lib = None


def lib(path: str | None = None):
    """Loads libdect.so (built by paper_1905_00934_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libdect.so not built ({p}); run __graft_entry__.build() first")
        L = ctypes.CDLL(p)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(status: int):
    if status != OK:
        raise DectError(status, lib().dect_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    """Data pointer of a torch tensor or numpy array (must be contiguous float32 unless noted)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(t.ctypes.data)
    assert t.is_contiguous(), "tensors passed to dect must be contiguous"
    return ctypes.c_void_p(t.data_ptr())


def version() -> str:
    return lib().dect_version().decode()


def sync(stream=None):
    _check(lib().dect_sync(_stream(stream)))


# ---- geometry / spectra -----------------------------------------------------------------------

def geom_desc(g) -> GeomDesc:
    """GeomDesc from any object with the synth.geometry.Geometry fields."""
    return GeomDesc(g.kind, g.nx, g.ny, g.n_views, g.n_bins, g.pixel_cm, g.angle0_rad, g.angle_span_rad,
                    g.bin_pitch_cm, g.bin_offset_cm, g.sod_cm, g.sdd_cm)


def geometry_create(g) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    d = geom_desc(g) if not isinstance(g, GeomDesc) else g
    _check(lib().dect_geometry_create(ctypes.byref(d), ctypes.byref(h)))
    return h


def geometry_destroy(h):
    lib().dect_geometry_destroy(h)


def spectra_create(S_h, S_l, f_kn, f_p) -> ctypes.c_void_p:
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (S_h, S_l, f_kn, f_p)]
    h = ctypes.c_void_p()
    _check(lib().dect_spectra_create(arrs[0].size, *[ctypes.c_void_p(a.ctypes.data) for a in arrs], ctypes.byref(h)))
    return h


def spectra_destroy(h):
    lib().dect_spectra_destroy(h)


# ---- operators ----------------------------------------------------------------------------------

def _dtype(t):
    import torch

    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError(f"dect supports float32 and float64 tensors, not {t.dtype}")


# Argument checks before a pointer reaches the library: the C entry points take plain pointers and
# trust their sizes, so a tensor of the wrong dtype, shape or device is refused here.
def _tensor(t, name, dtype=None, shape=None, numel=None, cuda=True):
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise TypeError(f"{name} must be {dtype}, not {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, not {tuple(t.shape)}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, not {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if cuda and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    return t


def _cuda(**tensors):
    """Every given tensor is a CUDA tensor, all on one device."""
    dev = None
    for name, t in tensors.items():
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if dev is None:
            dev = t.device
        elif t.device != dev:
            raise ValueError(f"{name} is on {t.device}, the other arrays on {dev}")


def _geom(geom):
    """(handle, (nx, ny, n_views, n_bins) or None): a solver.Geometry also gives its shape."""
    h = getattr(geom, "handle", geom)
    if all(hasattr(geom, k) for k in ("nx", "ny", "n_views", "n_bins")):
        return h, (geom.nx, geom.ny, geom.n_views, geom.n_bins)
    return h, None


def _pair(x, out, name_in, name_out, shape_in, shape_out, dtypes):
    """Checks an (input, output) pair of one dtype; shapes [nch, ...] with nch 1 or 2."""
    import torch

    _tensor(x, name_in, dtype=dtypes, cuda=False)
    if x.dim() != 3 or x.shape[0] not in (1, 2):
        raise ValueError(f"{name_in} must be [n_channels (1 or 2), ...], not {tuple(x.shape)}")
    _tensor(out, name_out, dtype=x.dtype, cuda=False)
    if out.dim() != 3 or out.shape[0] != x.shape[0]:
        raise ValueError(f"{name_out} must be [{x.shape[0]}, ...], not {tuple(out.shape)}")
    if shape_in is not None and tuple(x.shape[1:]) != tuple(shape_in):
        raise ValueError(f"{name_in} must be [n_channels, {shape_in[0]}, {shape_in[1]}], not {tuple(x.shape)}")
    if shape_out is not None and tuple(out.shape[1:]) != tuple(shape_out):
        raise ValueError(f"{name_out} must be [n_channels, {shape_out[0]}, {shape_out[1]}], not {tuple(out.shape)}")
    if not (x.is_cuda and out.is_cuda) or x.device != out.device:
        raise ValueError(f"{name_in} and {name_out} must be CUDA tensors on one device")


def project(geom, x, out, stream=None):
    """out[c] = R x[c]; x [nch, ny, nx], out [nch, n_views, n_bins] (CUDA float32 or float64, one dtype).
    geom is a geometry handle or a solver.Geometry; with the latter the shapes are checked too."""
    import torch

    h, dims = _geom(geom)
    _pair(x, out, "x", "out", None if dims is None else (dims[1], dims[0]),
          None if dims is None else (dims[2], dims[3]), (torch.float32, torch.float64))
    _check(lib().dect_project(h, x.shape[0], _dtype(x), _ptr(x), _ptr(out), _stream(stream)))
    return out


NOALLOC_SCRATCH_BYTES = 4 * 1024 * 1024


def project_noalloc(geom, x, out, stream=None):
    """Like project, but with the library's fixed scratch array instead of any allocation.

    For callers that must not allocate device memory (e.g. while a stream is being captured).
    Images must fit the fixed scratch (about 320 x 320); calls must not overlap on the GPU.
    geom is a geometry handle or a solver.Geometry; with the latter the shapes are checked too.
    x: float32 [nch, ny, nx], out: float32 [nch, n_views, n_bins] (CUDA, contiguous), nch 1 or 2.
    """
    import torch

    for name, t in (("x", x), ("out", out)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32:
            raise TypeError(f"project_noalloc: {name} must be a float32 tensor")
        if not t.is_cuda or t.dim() != 3 or not t.is_contiguous():
            raise ValueError(f"project_noalloc: {name} must be a contiguous 3-d CUDA tensor")
    if x.shape[0] not in (1, 2) or out.shape[0] != x.shape[0]:
        raise ValueError("project_noalloc: x and out need the same channel count, 1 or 2")
    handle = getattr(geom, "handle", geom)
    if hasattr(geom, "handle"):
        if tuple(x.shape[1:]) != (geom.ny, geom.nx) or tuple(out.shape[1:]) != (geom.n_views, geom.n_bins):
            raise ValueError(f"project_noalloc: shapes {tuple(x.shape)} -> {tuple(out.shape)} do not match the "
                             f"geometry ({geom.ny} x {geom.nx} image, {geom.n_views} x {geom.n_bins} sinogram)")
    _check(lib().dect_project_noalloc(handle, x.shape[0], _ptr(x), _ptr(out), _stream(stream)))
    return out


def backproject(geom, sino, out, stream=None):
    """out[c] = R^T sino[c] (exact adjoint of project); sino [nch, n_views, n_bins], out [nch, ny, nx]
    (CUDA float32 or float64, one dtype)."""
    import torch

    h, dims = _geom(geom)
    _pair(sino, out, "sino", "out", None if dims is None else (dims[2], dims[3]),
          None if dims is None else (dims[1], dims[0]), (torch.float32, torch.float64))
    _check(lib().dect_backproject(h, sino.shape[0], _dtype(sino), _ptr(sino), _ptr(out), _stream(stream)))
    return out


def decompose_rays(spec, m_h, m_l, w_h, w_l, v_c, v_p, rho_c, rho_p, iters, a_c, a_p, mu, status=None, stream=None):
    """Eq. 13 per ray; a_c, a_p, mu are updated in place (CUDA float32 arrays of one length; status uint8)."""
    import torch

    n = _tensor(a_c, "a_c", dtype=torch.float32, cuda=False).numel()
    for name, t in (("m_h", m_h), ("m_l", m_l), ("w_h", w_h), ("w_l", w_l), ("v_c", v_c), ("v_p", v_p),
                    ("a_p", a_p), ("mu", mu)):
        _tensor(t, name, dtype=torch.float32, numel=n, cuda=False)
    if status is not None:
        _tensor(status, "status", dtype=torch.uint8, numel=n, cuda=False)
    _cuda(m_h=m_h, m_l=m_l, w_h=w_h, w_l=w_l, v_c=v_c, v_p=v_p, a_c=a_c, a_p=a_p, mu=mu, status=status)
    _check(lib().dect_decompose_rays(spec, n, _ptr(m_h), _ptr(m_l), _ptr(w_h), _ptr(w_l), _ptr(v_c), _ptr(v_p),
                                     float(rho_c), float(rho_p), int(iters), _ptr(a_c), _ptr(a_p), _ptr(mu),
                                     _ptr(status), _stream(stream)))


def fbp(geom, sino, out, clamp_nonneg=False, stream=None):
    """out[c] = filtered backprojection of sino[c] (CUDA float32 [nch, V, Nb] -> [nch, ny, nx])."""
    import torch

    h, dims = _geom(geom)
    _pair(sino, out, "sino", "out", None if dims is None else (dims[2], dims[3]),
          None if dims is None else (dims[1], dims[0]), torch.float32)
    _check(lib().dect_fbp(h, sino.shape[0], _ptr(sino), _ptr(out), 1 if clamp_nonneg else 0, _stream(stream)))
    return out


def cdm_fbp(geom, spec, m_h, m_l, w_h, w_l, iters, out, work=None, stream=None):
    """CDM-FBP: per-ray decomposition with rho = 0, a >= 0, FBP of both bases into out [2, ny, nx]
    (CUDA float32; measurements [n_views, n_bins]; work None or 4 n_views n_bins floats)."""
    import torch

    h, dims = _geom(geom)
    n = None if dims is None else dims[2] * dims[3]
    _tensor(m_h, "m_h", dtype=torch.float32, numel=n, cuda=False)
    n = m_h.numel()
    for name, t in (("m_l", m_l), ("w_h", w_h), ("w_l", w_l)):
        _tensor(t, name, dtype=torch.float32, numel=n, cuda=False)
    _tensor(out, "out", dtype=torch.float32, shape=None if dims is None else (2, dims[1], dims[0]), cuda=False)
    if work is not None:
        _tensor(work, "work", dtype=torch.float32, numel=4 * n, cuda=False)
    _cuda(m_h=m_h, m_l=m_l, w_h=w_h, w_l=w_l, out=out, work=work)
    _check(lib().dect_cdm_fbp(h, spec, _ptr(m_h), _ptr(m_l), _ptr(w_h), _ptr(w_l), int(iters), _ptr(work),
                              _ptr(out), _stream(stream)))
    return out


def forward_model(spec, a_c, a_p, f_h=None, f_l=None, jac=None, stream=None):
    """Eq. 3 per ray (and its Jacobian [n, 4] if jac is given); CUDA arrays of one dtype (float32/float64)."""
    import torch

    n = _tensor(a_c, "a_c", dtype=(torch.float32, torch.float64), cuda=False).numel()
    _tensor(a_p, "a_p", dtype=a_c.dtype, numel=n, cuda=False)
    for name, t, k in (("f_h", f_h, n), ("f_l", f_l, n), ("jac", jac, 4 * n)):
        if t is not None:
            _tensor(t, name, dtype=a_c.dtype, numel=k, cuda=False)
    _cuda(a_c=a_c, a_p=a_p, f_h=f_h, f_l=f_l, jac=jac)
    _check(lib().dect_forward_model(spec, a_c.numel(), _dtype(a_c), _ptr(a_c), _ptr(a_p), _ptr(f_h), _ptr(f_l),
                                    _ptr(jac), _stream(stream)))


def forward_model_vjp(spec, a_c, a_p, g_h, g_l, grad_c, grad_p, stream=None):
    """Transpose of the forward model's Jacobian applied to (g_h, g_l); CUDA arrays of one dtype."""
    import torch

    n = _tensor(a_c, "a_c", dtype=(torch.float32, torch.float64), cuda=False).numel()
    for name, t in (("a_p", a_p), ("g_h", g_h), ("g_l", g_l), ("grad_c", grad_c), ("grad_p", grad_p)):
        _tensor(t, name, dtype=a_c.dtype, numel=n, cuda=False)
    _cuda(a_c=a_c, a_p=a_p, g_h=g_h, g_l=g_l, grad_c=grad_c, grad_p=grad_p)
    _check(lib().dect_forward_model_vjp(spec, a_c.numel(), _dtype(a_c), _ptr(a_c), _ptr(a_p), _ptr(g_h), _ptr(g_l),
                                        _ptr(grad_c), _ptr(grad_p), _stream(stream)))


# ---- ADMM solver ----------------------------------------------------------------------------------

def params_default(**kw) -> Params:
    """The library's defaults (the paper's parameters), with the given fields replaced; an unknown
    field name raises TypeError instead of being dropped."""
    fields = {f[0] for f in Params._fields_}
    unknown = sorted(set(kw) - fields)
    if unknown:
        raise TypeError(f"unknown solver parameter(s) {unknown}; the fields are {sorted(fields)}")
    p = Params()
    lib().dect_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def admm_create(geoms, spec, params: Params) -> ctypes.c_void_p:
    arr = (ctypes.c_void_p * len(geoms))(*[g.value if isinstance(g, ctypes.c_void_p) else g for g in geoms])
    h = ctypes.c_void_p()
    _check(lib().dect_admm_create(ctypes.cast(arr, ctypes.c_void_p), len(geoms), spec, ctypes.byref(params),
                                  ctypes.byref(h)))
    return h


def admm_destroy(h):
    lib().dect_admm_destroy(h)


def admm_set_data(h, slice_index, m_h, m_l, w_h, w_l, x0=None, stream=None, n_rays=None, n_pix=None):
    """Measurements float32 [n_views][n_bins] and an optional start image float32 [2][ny][nx], host or
    device (sizes checked when n_rays / n_pix are given)."""
    import torch

    n_rays = _tensor(m_h, "m_h", dtype=torch.float32, numel=n_rays, cuda=False).numel()
    for name, t in (("m_l", m_l), ("w_h", w_h), ("w_l", w_l)):
        _tensor(t, name, dtype=torch.float32, numel=n_rays, cuda=False)
    if x0 is not None:
        _tensor(x0, "x0", dtype=torch.float32, numel=None if n_pix is None else 2 * n_pix, cuda=False)
    _check(lib().dect_admm_set_data(h, slice_index, _ptr(m_h), _ptr(m_l), _ptr(w_h), _ptr(w_l), _ptr(x0),
                                    _stream(stream)))


def admm_set_truth(h, slice_index, truth, stream=None, n_pix=None):
    """Ground truth float32 [2][ny][nx], host or device."""
    import torch

    _tensor(truth, "truth", dtype=torch.float32, numel=None if n_pix is None else 2 * n_pix, cuda=False)
    _check(lib().dect_admm_set_truth(h, slice_index, _ptr(truth), _stream(stream)))


def admm_step(h, iters, stream=None):
    _check(lib().dect_admm_step(h, int(iters), _stream(stream)))


def reconstruct(h, iters, stream=None):
    _check(lib().dect_reconstruct(h, int(iters), _stream(stream)))


def admm_get(h, slice_index, which, out, stream=None):
    nbytes = out.numel() * out.element_size() if not isinstance(out, np.ndarray) else out.nbytes
    _check(lib().dect_admm_get(h, slice_index, which, _ptr(out), nbytes, _stream(stream)))
    return out


def admm_stats(h, slice_index, stream=None) -> dict:
    s = Stats()
    _check(lib().dect_admm_stats(h, slice_index, ctypes.byref(s), _stream(stream)))
    return {"iteration": s.iteration, "rho": list(s.rho), "r_pri": list(s.r_pri), "r_dual": list(s.r_dual),
            "xi_db": list(s.xi_db), "count_R": s.count_R, "count_RT": s.count_RT, "count_f": s.count_f,
            "count_launches": s.count_launches, "bp_view_groups": s.bp_view_groups, "objective": s.objective,
            "objective_iteration": s.objective_iteration, "bp_tile": s.bp_tile, "bp_cluster": s.bp_cluster,
            "bp_slices": s.bp_slices, "bp_reduce": s.bp_reduce, "proj_views": s.proj_views}


def admm_save(h, stream=None) -> np.ndarray:
    """The solver's state image (checkpoint) as a host uint8 array."""
    n = ctypes.c_size_t()
    _check(lib().dect_admm_state_bytes(h, ctypes.byref(n)))
    buf = np.empty(n.value, dtype=np.uint8)
    _check(lib().dect_admm_save(h, buf.ctypes.data, buf.nbytes, _stream(stream)))
    return buf


def admm_load(h, image, stream=None):
    """Restores a state image written by admm_save (host bytes-like or uint8 array)."""
    buf = np.ascontiguousarray(np.frombuffer(image, dtype=np.uint8) if not isinstance(image, np.ndarray) else image,
                               dtype=np.uint8)
    _check(lib().dect_admm_load(h, buf.ctypes.data, buf.nbytes, _stream(stream)))


PHASES = ["texture", "project", "backproject", "precond", "udm", "update", "reduce", "bp_finalize"]


def admm_profile(h, iters, stream=None):
    """Per-phase device milliseconds and kernel launches over `iters` profiled iterations."""
    ms = (ctypes.c_double * len(PHASES))()
    nl = (ctypes.c_int64 * len(PHASES))()
    _check(lib().dect_admm_profile(h, int(iters), _stream(stream), ms, nl))
    return {p: (ms[i], nl[i]) for i, p in enumerate(PHASES)}
