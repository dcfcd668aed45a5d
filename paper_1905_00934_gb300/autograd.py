"""torch.autograd wrappers over libdect (marshalling only; the arithmetic is in the CUDA kernels).

* project(x, geometry): R x (Eq. 2-3's projection matrix) with the R^T kernel as its
  backward pass. x has any leading dims [..., ny, nx]; float32 or float64 on the GPU.
* forward_model(a_c, a_p, spectra): f_h, f_l of Eq. 3 per ray, whose backward is the transpose
  of the per-ray 2x2 Jacobian (the derivative the decomposition step of Eq. 13 linearises).

Composing them gives the gradient of any loss of the measurements model f(R x), e.g. the
weighted data fidelity 1/2 ||f(R x) - m||^2_Sigma of Eq. 4.
"""
from __future__ import annotations

import torch

from . import dect


def _chunks(n):
    for c0 in range(0, n, 2):
        yield c0, min(n, c0 + 2)


class _Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, geometry):
        ctx.geometry = geometry
        g = geometry
        lead = x.shape[:-2]
        xf = x.reshape(-1, g.ny, g.nx).contiguous()
        out = torch.empty((xf.shape[0], g.n_views, g.n_bins), dtype=x.dtype, device=x.device)
        for a, b in _chunks(xf.shape[0]):
            dect.project(g, xf[a:b], out[a:b])
        return out.reshape(*lead, g.n_views, g.n_bins)

    @staticmethod
    def backward(ctx, grad):
        g = ctx.geometry
        lead = grad.shape[:-2]
        gf = grad.reshape(-1, g.n_views, g.n_bins).contiguous()
        out = torch.empty((gf.shape[0], g.ny, g.nx), dtype=grad.dtype, device=grad.device)
        for a, b in _chunks(gf.shape[0]):
            dect.backproject(g, gf[a:b], out[a:b])
        return out.reshape(*lead, g.ny, g.nx), None


def project(x: torch.Tensor, geometry) -> torch.Tensor:
    """Differentiable forward projection; geometry is a paper_1905_00934_gb300.Geometry."""
    return _Project.apply(x, geometry)


class _ForwardModel(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a_c, a_p, spectra):
        a_c = a_c.contiguous()
        a_p = a_p.contiguous()
        f_h = torch.empty_like(a_c)
        f_l = torch.empty_like(a_c)
        dect.forward_model(spectra.handle, a_c, a_p, f_h, f_l)
        ctx.spectra = spectra
        ctx.save_for_backward(a_c, a_p)
        return f_h, f_l

    @staticmethod
    def backward(ctx, g_h, g_l):
        a_c, a_p = ctx.saved_tensors
        g_h = torch.zeros_like(a_c) if g_h is None else g_h.contiguous()
        g_l = torch.zeros_like(a_c) if g_l is None else g_l.contiguous()
        grad_c = torch.empty_like(a_c)
        grad_p = torch.empty_like(a_c)
        dect.forward_model_vjp(ctx.spectra.handle, a_c, a_p, g_h, g_l, grad_c, grad_p)
        return grad_c, grad_p, None


def forward_model(a_c: torch.Tensor, a_p: torch.Tensor, spectra):
    """Differentiable f_h, f_l of Eq. 3 per ray; spectra is a paper_1905_00934_gb300.Spectra."""
    return _ForwardModel.apply(a_c, a_p, spectra)
