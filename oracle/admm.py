"""One ADMM iteration of UDM(m)-PCG(n) (Sec. 3.3), FP64, with its pieces.

TEST INFRASTRUCTURE ONLY. Plain numpy; the projector pair and the per-ray
decomposition come from oracle.projector / oracle.spectral (C, FP64).

Notation follows the paper: basis beta in {c, p} (index 0 = Compton, 1 = PE);
x_beta the image, a_beta = R x_beta the new auxiliary (measurement fitting as a
constraint, Sec. 3.3), y_beta = D x_beta (TV split), z_beta = x_beta
(non-negativity split), u^a, u^y, u^z the scaled duals, rho_beta the penalty.
Arrays carry the basis as their leading axis.

Readings where the paper is silent (each listed in the design notes):
  * D: forward differences along x (columns) and y (rows), the difference at
    the last column/row is 0; anisotropic TV, so y holds two components.
  * shrinkage (Eq. 9): soft threshold sign(t) max(|t| - tau, 0).
  * preconditioner (Sec. 3.3, "high-passing filter"): a circulant model of the
    Eq. 12 operator R^T R + D^T D + I, H = 1 / (Re F[R^T R delta] + |F[D]|^2 + 1)
    on a zero-padded grid (power of two >= 2N per axis), F[R^T R delta] the DFT
    of the point response at the centre pixel (clamped >= 0). At low frequency
    R^T R ~ 1/|w|, so H behaves as the ramp filter the paper names. The plain ramp filter
    1 / (K/|w| + 1) is the alternative (PRECOND_RAMP), for the preconditioner comparison.
  * adaptive rho (Boyd et al. 2011, Sec. 3.4.1): mu_b = 10, tau = 2, per basis,
    r_pri = ||[a; y; z] - [R; D; I] x||, r_dual = rho ||[a; y; z]_new - [a; y; z]_old||;
    when rho changes the scaled duals are divided by the same factor.
  * order within an iteration: x (Eq. 12) -> a (Eq. 13) -> y, z (Eq. 9-10) ->
    u (Eq. 11 with the a-block) -> rho.
  * R x is carried: PCG updates it as R x += alpha R p, so one iteration costs
    2n applications of R and 2(n+1) of R^T over the two bases (Table 1).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import fbp, projector, spectral


# ----------------------------------------------------------------------------
# finite differences (Eq. 5's D) and the element-wise updates (Eq. 9-11)

def grad(x: np.ndarray) -> np.ndarray:
    """D x for an image [ny][nx] -> [2][ny][nx] (component 0: along x, 1: along y)."""
    out = np.zeros((2,) + x.shape)
    out[0, :, :-1] = x[:, 1:] - x[:, :-1]
    out[1, :-1, :] = x[1:, :] - x[:-1, :]
    return out


def grad_t(y: np.ndarray) -> np.ndarray:
    """D^T y, the adjoint of grad."""
    out = np.zeros(y.shape[1:])
    out[:, :-1] -= y[0, :, :-1]
    out[:, 1:] += y[0, :, :-1]
    out[:-1, :] -= y[1, :-1, :]
    out[1:, :] += y[1, :-1, :]
    return out


def shrinkage(t: np.ndarray, tau: float) -> np.ndarray:
    """Eq. 9's shrinkage: sign(t) max(|t| - tau, 0)."""
    return np.sign(t) * np.maximum(np.abs(t) - tau, 0.0)


def xi_db(x: np.ndarray, truth: np.ndarray) -> float:
    """Eq. 14: 20 log10(||x - x*|| / ||x*||)."""
    return float(20.0 * np.log10(np.linalg.norm(x - truth) / np.linalg.norm(truth)))


# ----------------------------------------------------------------------------
# preconditioner (Sec. 3.3)

PRECOND_NONE, PRECOND_CIRCULANT, PRECOND_RAMP = 0, 1, 2
INIT_PCG, INIT_CDM_FBP = 0, 1


def pad_size(n: int) -> int:
    p = 1
    while p < 2 * n:
        p *= 2
    return p


def point_response(geom) -> np.ndarray:
    """R^T R applied to a unit impulse at pixel (ny//2, nx//2)."""
    d = np.zeros((geom.ny, geom.nx))
    d[geom.ny // 2, geom.nx // 2] = 1.0
    return projector.backproject(geom, projector.project(geom, d))


def point_response_dft(geom) -> np.ndarray:
    """Re F[R^T R delta] on the [Py][Px] padded grid, the point response centred at grid index
    (0, 0) (wrapped), clamped >= 0."""
    py, px = pad_size(geom.ny), pad_size(geom.nx)
    psf = point_response(geom)
    grid = np.zeros((py, px))
    jj = (np.arange(geom.ny) - geom.ny // 2) % py
    ii = (np.arange(geom.nx) - geom.nx // 2) % px
    grid[np.ix_(jj, ii)] = psf
    return np.maximum(np.fft.fft2(grid).real, 0.0)


def precond_response(geom, with_grad: bool = True) -> np.ndarray:
    """H on the [Py][Px] padded frequency grid (real, > 0)."""
    phat = point_response_dft(geom)
    py, px = phat.shape
    wy = 2.0 * np.pi * np.arange(py) / py
    wx = 2.0 * np.pi * np.arange(px) / px
    dhat = 4.0 * np.sin(wy / 2.0)[:, None] ** 2 + 4.0 * np.sin(wx / 2.0)[None, :] ** 2
    return 1.0 / (phat + (dhat if with_grad else 0.0) + 1.0)


def ramp_response(geom) -> np.ndarray:
    """The plain ramp filter as the preconditioner (Sec. 3.3 names a ramp / high-pass filter):
    R^T R replaced by its asymptotic form K / |w| and D^T D dropped, H = 1 / (K / |w| + 1) =
    |w| / (K + |w|). |w| is the wrapped radial frequency in radians per pixel, floored at the
    first non-zero grid frequency 2 pi / max(Px, Py) so that H(0) > 0. K is read off the point
    response at w = (0, pi/4): K = (pi/4) Re F[R^T R delta](0, Px/8)."""
    phat = point_response_dft(geom)
    py, px = phat.shape
    K = phat[0, px // 8] * (np.pi / 4.0)
    ky, kx = np.arange(py), np.arange(px)
    wy = 2.0 * np.pi * np.minimum(ky, py - ky) / py
    wx = 2.0 * np.pi * np.minimum(kx, px - kx) / px
    w = np.maximum(np.hypot(wy[:, None], wx[None, :]), 2.0 * np.pi / max(px, py))
    return 1.0 / (K / w + 1.0)


def apply_precond(H: np.ndarray, r: np.ndarray) -> np.ndarray:
    """M^{-1} r = crop(IDFT(H * DFT(zero-pad(r))))."""
    ny, nx = r.shape
    buf = np.zeros(H.shape)
    buf[:ny, :nx] = r
    return np.fft.ifft2(H * np.fft.fft2(buf)).real[:ny, :nx]


# ----------------------------------------------------------------------------
# problem, parameters and state

@dataclasses.dataclass
class Params:
    lam: tuple = (1e-5, 1e-5)          # lambda_c, lambda_p (Sec. 4)
    rho0: tuple = (1e-3, 1e-3)         # initial rho_c, rho_p (Sec. 4)
    m_udm: int = 1                     # LM iterations per ADMM iteration (UDM(m))
    n_pcg: int = 1                     # CG iterations per ADMM iteration (PCG(n))
    mu_b: float = 10.0                 # residual-balancing threshold
    tau: float = 2.0                   # residual-balancing factor
    lm_mu0: float = 1e-3               # initial LM damping
    adapt_rho: bool = True
    precondition: int = 1              # PRECOND_NONE (plain CG), PRECOND_CIRCULANT or PRECOND_RAMP
    # initialisation
    kappa: float = 1e-2                # x_p0 = kappa * x_c0
    init_udm_iters: int = 10
    init_pcg_iters: int = 10
    init: int = 0                      # INIT_PCG (the stand-in below) or INIT_CDM_FBP (the paper's start)


@dataclasses.dataclass
class Counters:
    """Operator applications, counted per basis (Table 1's units)."""
    R: int = 0
    RT: int = 0
    f: int = 0   # evaluations of f per ray (f_h and f_l at one point count as 2)


class Problem:
    def __init__(self, geom, spec, m_h, m_l, w_h, w_l, params: Params):
        self.geom = geom
        self.spec = spec
        self.m_h = np.asarray(m_h, dtype=np.float64).reshape(geom.n_views, geom.n_bins)
        self.m_l = np.asarray(m_l, dtype=np.float64).reshape(geom.n_views, geom.n_bins)
        self.w_h = np.asarray(w_h, dtype=np.float64).reshape(geom.n_views, geom.n_bins)
        self.w_l = np.asarray(w_l, dtype=np.float64).reshape(geom.n_views, geom.n_bins)
        self.params = params
        mode = int(params.precondition)
        if mode not in (PRECOND_NONE, PRECOND_CIRCULANT, PRECOND_RAMP):
            raise ValueError(f"precondition must be 0, 1 or 2, got {params.precondition}")
        self.H = self.H_init = None
        if mode == PRECOND_CIRCULANT:
            self.H, self.H_init = precond_response(geom, True), precond_response(geom, False)
        elif mode == PRECOND_RAMP:
            self.H = self.H_init = ramp_response(geom)
        self.count = Counters()

    # operators on both bases, with Table 1 counting
    def R(self, x2):
        self.count.R += 2
        return np.stack([projector.project(self.geom, x2[b]) for b in (0, 1)])

    def RT(self, s2):
        self.count.RT += 2
        return np.stack([projector.backproject(self.geom, s2[b]) for b in (0, 1)])

    def M(self, r2, H):
        if H is None:
            return r2.copy()
        return np.stack([apply_precond(H, r2[b]) for b in (0, 1)])


@dataclasses.dataclass
class State:
    x: np.ndarray      # [2][ny][nx]
    Rx: np.ndarray     # [2][V][Nb]
    a: np.ndarray      # [2][V][Nb]
    ua: np.ndarray     # [2][V][Nb]
    y: np.ndarray      # [2][2][ny][nx]
    uy: np.ndarray     # [2][2][ny][nx]
    z: np.ndarray      # [2][ny][nx]
    uz: np.ndarray     # [2][ny][nx]
    rho: np.ndarray    # [2]
    mu: np.ndarray     # [V][Nb]  LM damping per ray
    status: np.ndarray  # [V][Nb] uint8
    r_pri: np.ndarray = None
    r_dual: np.ndarray = None
    iteration: int = 0

    def copy(self):
        return State(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in dataclasses.asdict(self).items()})


def state_from_image(prob: Problem, x0_c, x0_p) -> State:
    """ADMM start from an image: R x0, a = R x0, y = D x0, z = x0, zero duals."""
    g = prob.geom
    x = np.stack([np.asarray(x0_c, dtype=np.float64).reshape(g.ny, g.nx),
                  np.asarray(x0_p, dtype=np.float64).reshape(g.ny, g.nx)])
    Rx = prob.R(x)
    y = np.stack([grad(x[b]) for b in (0, 1)])
    return State(x=x, Rx=Rx, a=Rx.copy(), ua=np.zeros_like(Rx), y=y, uy=np.zeros_like(y),
                 z=x.copy(), uz=np.zeros_like(x), rho=np.array(prob.params.rho0, dtype=np.float64),
                 mu=np.full((g.n_views, g.n_bins), prob.params.lm_mu0),
                 status=np.zeros((g.n_views, g.n_bins), dtype=np.uint8))


# ----------------------------------------------------------------------------
# Eq. 12: the x-update by n PCG iterations (both bases; they are independent)

def pcg_x_update(prob: Problem, st: State, n: int, with_grad: bool = True, H=None):
    """Warm-started PCG on (R^T R + D^T D + I) x = R^T(a+u^a) + D^T(y+u^y) + (z+u^z).

    Residual form: r0 = R^T(a + u^a - R x) + D^T(y + u^y - D x) + (z + u^z - x).
    R x is carried in st.Rx and updated with alpha R p. Returns the alphas.
    with_grad=False drops the D block (used by the initialisation).
    """
    x, Rx = st.x, st.Rx
    r = prob.RT(st.a + st.ua - Rx) + (st.z + st.uz - x)
    if with_grad:
        r += np.stack([grad_t(st.y[b] + st.uy[b] - grad(x[b])) for b in (0, 1)])
    s = prob.M(r, H)
    p = s.copy()
    rs = np.array([np.vdot(r[b], s[b]) for b in (0, 1)])
    alphas = []
    for it in range(n):
        q = prob.R(p)
        Ap = prob.RT(q) + p
        if with_grad:
            Ap += np.stack([grad_t(grad(p[b])) for b in (0, 1)])
        pAp = np.array([np.vdot(p[b], Ap[b]) for b in (0, 1)])
        alpha = np.where(pAp > 0, rs / np.where(pAp > 0, pAp, 1.0), 0.0)
        x = x + alpha[:, None, None] * p
        Rx = Rx + alpha[:, None, None] * q
        alphas.append(alpha)
        if it == n - 1:
            break
        r = r - alpha[:, None, None] * Ap
        s = prob.M(r, H)
        rs_new = np.array([np.vdot(r[b], s[b]) for b in (0, 1)])
        beta = np.where(rs > 0, rs_new / np.where(rs > 0, rs, 1.0), 0.0)
        p = s + beta[:, None, None] * p
        rs = rs_new
    st.x, st.Rx = x, Rx
    return alphas


# ----------------------------------------------------------------------------
# residual balancing (Sec. 3.2, following Boyd et al. 2011, Sec. 3.4.1)

def residual_balance(st: State, P: Params, a_old, y_old, z_old, Dx, a_block: bool = True) -> None:
    """Residuals and the adaptive penalty, in place on the state after the dual update.

    Per basis b: r_pri = ||[a; y; z] - [R x; D x; x]||, r_dual = rho ||[a; y; z] - [a; y; z]_old||
    (the surrogate without the C^T factor). If r_pri > mu_b r_dual, rho grows by tau; else if
    r_dual > mu_b r_pri it shrinks by tau. The scaled duals u = y_dual / rho follow: they are
    divided by the factor rho was multiplied by, so the unscaled duals stay put.
    a_block=False drops the a terms and leaves u^a alone (the LM x CG splitting has no a-block).
    """
    r_pri = np.zeros(2)
    r_dual = np.zeros(2)
    for b in (0, 1):
        pri_a = np.sum((st.a[b] - st.Rx[b]) ** 2) if a_block else 0.0
        dual_a = np.sum((st.a[b] - a_old[b]) ** 2) if a_block else 0.0
        r_pri[b] = np.sqrt(pri_a + np.sum((st.y[b] - Dx[b]) ** 2) + np.sum((st.z[b] - st.x[b]) ** 2))
        r_dual[b] = st.rho[b] * np.sqrt(dual_a + np.sum((st.y[b] - y_old[b]) ** 2)
                                        + np.sum((st.z[b] - z_old[b]) ** 2))
    st.r_pri, st.r_dual = r_pri, r_dual
    if P.adapt_rho:
        for b in (0, 1):
            factor = 1.0
            if r_pri[b] > P.mu_b * r_dual[b]:
                factor = P.tau
            elif r_dual[b] > P.mu_b * r_pri[b]:
                factor = 1.0 / P.tau
            if factor != 1.0:
                st.rho[b] *= factor
                if a_block:
                    st.ua[b] /= factor
                st.uy[b] /= factor
                st.uz[b] /= factor


# ----------------------------------------------------------------------------
# one ADMM iteration (Sec. 3.3)

def admm_iteration(prob: Problem, st: State) -> State:
    P = prob.params
    st = st.copy()
    a_old, y_old, z_old = st.a.copy(), st.y.copy(), st.z.copy()

    # Eq. 12
    pcg_x_update(prob, st, P.n_pcg, True, prob.H)

    # Eq. 13, with v_beta = R x_beta - u^a_beta
    v = st.Rx - st.ua
    ac, ap, mu, status = spectral.udm(prob.spec, prob.m_h, prob.m_l, prob.w_h, prob.w_l, v[0], v[1],
                                      st.rho[0], st.rho[1], P.m_udm, st.a[0], st.a[1], st.mu)
    prob.count.f += 4 * P.m_udm
    g = prob.geom
    st.a = np.stack([ac.reshape(g.n_views, g.n_bins), ap.reshape(g.n_views, g.n_bins)])
    st.mu = mu.reshape(g.n_views, g.n_bins)
    st.status = status.reshape(g.n_views, g.n_bins)

    # Eq. 9-10
    Dx = np.stack([grad(st.x[b]) for b in (0, 1)])
    st.y = np.stack([shrinkage(Dx[b] - st.uy[b], P.lam[b] / st.rho[b]) for b in (0, 1)])
    st.z = np.maximum(0.0, st.x - st.uz)

    # Eq. 11 with the a-block
    st.ua = st.ua + st.a - st.Rx
    st.uy = st.uy + st.y - Dx
    st.uz = st.uz + st.z - st.x

    # residuals and adaptive rho
    residual_balance(st, P, a_old, y_old, z_old, Dx)
    st.iteration += 1
    return st


# ----------------------------------------------------------------------------
# initialisation (Sec. 4: a Compton estimate, PE = scaled Compton)

def initial_image(prob: Problem):
    """x0 = (x_c0, kappa * x_c0).

    The paper starts from a CDM decomposition + FBP Compton image and a scaled
    copy for PE (params.init = INIT_CDM_FBP). Default stand-in (INIT_PCG, chosen
    before CDM-FBP existed here and kept as the default): a0 = per-ray decomposition (Eq. 13) with rho_c = 0,
    rho_p = rho0_p, v = 0, from a_c = m_l / sum_E S_l f_KN, a_p = 0; then
    x_c0 = max(0, PCG iterations on (R^T R + I) x = R^T a_c0 from 0).
    """
    P = prob.params
    g = prob.geom
    spec = prob.spec
    if P.init == INIT_CDM_FBP:
        # the paper's start: the Compton image of CDM-FBP (oracle.fbp), clamped, and a scaled copy
        ac, _ = fbp.cdm(spec, prob.m_h, prob.m_l, prob.w_h, prob.w_l, P.init_udm_iters, P.lm_mu0)
        prob.count.f += 4 * P.init_udm_iters
        xc = np.maximum(fbp.fbp(g, ac), 0.0)
        return xc, P.kappa * xc
    sl = spec.s_low / spec.s_low.sum()
    a_c0 = prob.m_l / float(np.dot(sl, spec.f_kn))
    zeros = np.zeros_like(prob.m_l)
    mu = np.full(zeros.shape, P.lm_mu0)
    ac, ap, _, _ = spectral.udm(spec, prob.m_h, prob.m_l, prob.w_h, prob.w_l, zeros, zeros,
                                0.0, P.rho0[1], P.init_udm_iters, a_c0, zeros, mu)
    prob.count.f += 4 * P.init_udm_iters
    a = np.stack([ac.reshape(zeros.shape), np.zeros_like(zeros)])
    x = np.zeros((2, g.ny, g.nx))
    st = State(x=x, Rx=np.zeros_like(a), a=a, ua=np.zeros_like(a), y=np.zeros((2, 2, g.ny, g.nx)),
               uy=np.zeros((2, 2, g.ny, g.nx)), z=np.zeros_like(x), uz=np.zeros_like(x),
               rho=np.array(P.rho0, dtype=np.float64), mu=mu, status=np.zeros(zeros.shape, np.uint8))
    pcg_x_update(prob, st, P.init_pcg_iters, with_grad=False, H=prob.H_init)
    xc = np.maximum(st.x[0], 0.0)
    return xc, P.kappa * xc


# ----------------------------------------------------------------------------
# monitors

def map_objective(prob: Problem, x2: np.ndarray) -> float:
    """Eq. 4 without g: 1/2 ||f(R x) - m||^2_Sigma + sum_beta lambda_beta |D x_beta|_1 (R x recomputed)."""
    Rx = np.stack([projector.project(prob.geom, x2[b]) for b in (0, 1)])
    fh, fl = spectral.forward_model(prob.spec, Rx[0], Rx[1])
    data = 0.5 * np.sum(prob.w_h.ravel() * (fh - prob.m_h.ravel()) ** 2 + prob.w_l.ravel() * (fl - prob.m_l.ravel()) ** 2)
    tv = sum(prob.params.lam[b] * np.abs(grad(x2[b])).sum() for b in (0, 1))
    return float(data + tv)


def run(prob: Problem, st: State, iters: int, truth=None, log=None):
    """iters ADMM iterations; optionally records xi (Eq. 14) per iteration."""
    hist = []
    for _ in range(iters):
        st = admm_iteration(prob, st)
        if truth is not None:
            hist.append((xi_db(st.x[0], truth[0]), xi_db(st.x[1], truth[1])))
        if log is not None:
            log(st)
    return st, hist
