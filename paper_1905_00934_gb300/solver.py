"""Handle-owning wrappers around the dect C ABI (marshalling only; every step runs in libdect)."""
from __future__ import annotations

import torch

from . import dect


class Geometry:
    """A dect geometry handle (the projection matrix R) built from a geometry description."""

    def __init__(self, g):
        self.desc = g
        self.handle = dect.geometry_create(g)
        self.nx, self.ny, self.n_views, self.n_bins = g.nx, g.ny, g.n_views, g.n_bins

    def project(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        squeeze = x.dim() == 2
        x = x.reshape(-1, self.ny, self.nx)
        if out is None:
            out = torch.empty((x.shape[0], self.n_views, self.n_bins), device=x.device, dtype=x.dtype)
        dect.project(self, x, out, stream)
        return out[0] if squeeze else out

    def backproject(self, s: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        squeeze = s.dim() == 2
        s = s.reshape(-1, self.n_views, self.n_bins)
        if out is None:
            out = torch.empty((s.shape[0], self.ny, self.nx), device=s.device, dtype=s.dtype)
        dect.backproject(self, s, out, stream)
        return out[0] if squeeze else out

    def fbp(self, s: torch.Tensor, out: torch.Tensor | None = None, clamp_nonneg: bool = False,
            stream=None) -> torch.Tensor:
        """Filtered backprojection of float32 sinograms [nch, V, Nb] (or [V, Nb])."""
        squeeze = s.dim() == 2
        s = s.reshape(-1, self.n_views, self.n_bins)
        if out is None:
            out = torch.empty((s.shape[0], self.ny, self.nx), device=s.device, dtype=torch.float32)
        dect.fbp(self, s, out, clamp_nonneg, stream)
        return out[0] if squeeze else out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and dect._lib is not None:
            dect.geometry_destroy(h)
            self.handle = None


def cdm_fbp(geo: Geometry, spec: "Spectra", m_h, m_l, w_h, w_l, iters: int = 20, work=None, stream=None):
    """The CDM-FBP comparison method: [2, ny, nx] (Compton, PE). work, if given, is a float32 device
    tensor of 4 V Nb elements and holds the per-ray line integrals (a_c, a_p) on return."""
    out = torch.empty((2, geo.ny, geo.nx), device=m_h.device, dtype=torch.float32)
    dect.cdm_fbp(geo, spec.handle, m_h, m_l, w_h, w_l, iters, out, work, stream)
    return out


class Spectra:
    """Spectral tables of Eq. 1-3 on the device."""

    def __init__(self, S_h, S_l, f_kn, f_p):
        self.handle = dect.spectra_create(S_h, S_l, f_kn, f_p)

    @classmethod
    def from_tables(cls, t):
        return cls(t.s_high, t.s_low, t.f_kn, t.f_p)

    def decompose(self, m_h, m_l, w_h, w_l, v_c, v_p, rho_c, rho_p, iters, a_c, a_p, mu, status=None, stream=None):
        dect.decompose_rays(self.handle, m_h, m_l, w_h, w_l, v_c, v_p, rho_c, rho_p, iters, a_c, a_p, mu, status,
                            stream)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and dect._lib is not None:
            dect.spectra_destroy(h)
            self.handle = None


class Solver:
    """ADMM solver over a batch of slices (UDM(m)-PCG(n), one CUDA graph per iteration)."""

    def __init__(self, geoms, spectra: Spectra, **params):
        self.geoms = list(geoms)
        self.spectra = spectra
        self.params = dect.params_default(**params)
        self.handle = dect.admm_create([g.handle for g in self.geoms], spectra.handle, self.params)

    def set_data(self, b, m_h, m_l, w_h, w_l, x0=None, stream=None):
        g = self.geoms[b]
        dect.admm_set_data(self.handle, b, m_h, m_l, w_h, w_l, x0, stream, n_rays=g.n_views * g.n_bins,
                           n_pix=g.nx * g.ny)

    def set_truth(self, b, truth, stream=None):
        g = self.geoms[b]
        dect.admm_set_truth(self.handle, b, truth, stream, n_pix=g.nx * g.ny)

    def step(self, iters=1, stream=None):
        dect.admm_step(self.handle, iters, stream)

    def reconstruct(self, iters, stream=None):
        dect.reconstruct(self.handle, iters, stream)

    def get(self, b, which, device="cuda", stream=None) -> torch.Tensor:
        g = self.geoms[b]
        shapes = {dect.X: (2, g.ny, g.nx), dect.RX: (2, g.n_views, g.n_bins), dect.A: (2, g.n_views, g.n_bins),
                  dect.UA: (2, g.n_views, g.n_bins), dect.Y: (2, 2, g.ny, g.nx), dect.UY: (2, 2, g.ny, g.nx),
                  dect.Z: (2, g.ny, g.nx), dect.UZ: (2, g.ny, g.nx), dect.MU: (g.n_views, g.n_bins)}
        if which == dect.H:
            py = 1
            while py < 2 * g.ny:
                py *= 2
            px = 1
            while px < 2 * g.nx:
                px *= 2
            shape = (py, px)
        else:
            shape = shapes[which]
        # float64 storage keeps (and returns) every array in float64
        dtype = torch.float64 if self.params.storage == dect.STORE_F64 else torch.float32
        out = torch.empty(shape, dtype=dtype, device=device)
        dect.admm_get(self.handle, b, which, out, stream)
        return out

    def profile(self, iters=1, stream=None) -> dict:
        return dect.admm_profile(self.handle, iters, stream)

    def stats(self, b=0, stream=None) -> dict:
        return dect.admm_stats(self.handle, b, stream)

    def save(self, stream=None):
        """Checkpoint: the solver's state as a host uint8 array (numpy)."""
        return dect.admm_save(self.handle, stream)

    def load(self, image, stream=None):
        """Resume from a checkpoint of a solver with the same slice shapes, storage and scheme."""
        dect.admm_load(self.handle, image, stream)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and dect._lib is not None:
            dect.admm_destroy(h)
            self.handle = None
