"""One ADMM iteration of the comparison scheme LM(m) x CG(n) (Sec. 3.2, Eq. 6-11; Table 1), FP64.

TEST INFRASTRUCTURE ONLY. Plain numpy on top of the oracle's projector pair and forward model.

The augmented Lagrangian of Eq. 6 splits only the TV and non-negativity terms (y = D x, z = x);
the measurement term stays inside the x-updates, which are two nonlinear least-squares problems
solved in turn by Levenberg-Marquardt (Eq. 7 for x_c with x_p fixed, then Eq. 8 for x_p with the
new x_c), each LM step solving its linear system by n plain CG iterations. Then y, z (Eq. 9-10),
the duals (Eq. 11 without an a-block) and rho (residual balancing) as in the new scheme.

Readings where the paper is silent (each listed in the design notes):
  * LM model: Gauss-Newton for the data term of basis beta around the current x,
        1/2 ||f(R x) - m||^2_Sigma ~ const + <e, R d> + 1/2 <R d, diag(g) R d>,
    e = w_h r_h J_h,beta + w_l r_l J_l,beta and g = w_h J_h,beta^2 + w_l J_l,beta^2 per ray
    (r = f - m, J the per-ray Jacobian of f), plus the augmented-Lagrangian term of basis beta,
    rho/2 ||[y; z] - C x + u||^2 with C = [D; I], which is quadratic.
  * damping: the Gauss-Newton data block is scaled by (1 + mu_beta) (Marquardt scaling of the data
    curvature), one mu per basis, mu0 = 1e-3, divided by 10 after an accepted step and multiplied
    by 10 after a rejected one, clamped to [1e-10, 1e10]; accept iff the basis' subproblem
    objective (data term + augmented-Lagrangian term) strictly decreases.
  * linear solve: n CG iterations (unpreconditioned: the paper's "CG") from d = 0 on
        ((1 + mu) R^T diag(g) R + rho (D^T D + I)) d = -(R^T e + rho C^T (C x - [y; z] - u)).
  * one LM step applies R^T once for the gradient, R and R^T once per CG iteration and R once
    for the trial point: (n + 1) of each per basis (Table 1's 2m(n+1) over both bases), and
    evaluates f twice (with the Jacobian at x, without it at the trial point: 4m over both).
"""
from __future__ import annotations

import numpy as np

from . import projector, spectral
from .admm import Problem, State, grad, grad_t, residual_balance, shrinkage, state_from_image


def _data_terms(prob: Problem, Rx: np.ndarray, jacobian: bool):
    """Per-ray residuals r_h, r_l (f - m) and, with jacobian, J = [dfh/dac, dfh/dap, dfl/dac, dfl/dap]."""
    out = spectral.forward_model(prob.spec, Rx[0], Rx[1], jacobian=jacobian)
    rh = out[0] - prob.m_h.ravel()
    rl = out[1] - prob.m_l.ravel()
    return (rh, rl, out[2]) if jacobian else (rh, rl)


def _data_cost(prob: Problem, rh, rl) -> float:
    return 0.5 * float(np.sum(prob.w_h.ravel() * rh * rh + prob.w_l.ravel() * rl * rl))


def _al_cost(rho: float, x, t, s) -> float:
    """rho/2 ||[y; z] - C x + u||^2 with t = y + u^y, s = z + u^z."""
    return 0.5 * rho * float(np.sum((t - grad(x)) ** 2) + np.sum((s - x) ** 2))


def lm_step(prob: Problem, st: State, b: int, n: int) -> bool:
    """One LM iteration on basis b (the other basis fixed); updates st.x[b], st.Rx[b], st.mu_x[b].
    Returns whether the step was accepted."""
    g = prob.geom
    rho = float(st.rho[b])
    mu = float(st.mu_x[b])
    x = st.x[b]
    t = st.y[b] + st.uy[b]
    s = st.z[b] + st.uz[b]

    rh, rl, J = _data_terms(prob, st.Rx, True)
    prob.count.f += 1
    jh, jl = J[:, b], J[:, 2 + b]
    wh, wl = prob.w_h.ravel(), prob.w_l.ravel()
    e = (wh * rh * jh + wl * rl * jl).reshape(g.n_views, g.n_bins)
    gw = (wh * jh * jh + wl * jl * jl).reshape(g.n_views, g.n_bins)
    cost0 = _data_cost(prob, rh, rl) + _al_cost(rho, x, t, s)

    # gradient of the subproblem objective at x
    gr = projector.backproject(g, e) + rho * (grad_t(grad(x) - t) + (x - s))
    prob.count.RT += 1

    # n CG iterations on ((1 + mu) R^T diag(g) R + rho (D^T D + I)) d = -gr, from d = 0
    d = np.zeros_like(x)
    r = -gr
    p = r.copy()
    rr = float(np.vdot(r, r))
    for _ in range(n):
        q = projector.project(g, p)
        prob.count.R += 1
        Ap = (1.0 + mu) * projector.backproject(g, gw * q) + rho * (grad_t(grad(p)) + p)
        prob.count.RT += 1
        pAp = float(np.vdot(p, Ap))
        if not pAp > 0.0:
            break
        alpha = rr / pAp
        d = d + alpha * p
        r = r - alpha * Ap
        rr_new = float(np.vdot(r, r))
        p = r + (rr_new / rr if rr > 0 else 0.0) * p
        rr = rr_new

    # trial point
    Rd = projector.project(g, d)
    prob.count.R += 1
    Rx1 = st.Rx.copy()
    Rx1[b] = Rx1[b] + Rd
    rh1, rl1 = _data_terms(prob, Rx1, False)
    prob.count.f += 1
    cost1 = _data_cost(prob, rh1, rl1) + _al_cost(rho, x + d, t, s)
    accepted = bool(np.isfinite(cost1) and cost1 < cost0)
    if accepted:
        st.x[b] = x + d
        st.Rx = Rx1
        mu *= 0.1
    else:
        mu *= 10.0
    st.mu_x[b] = min(max(mu, 1e-10), 1e10)
    return accepted


def lmcg_state(prob: Problem, x0_c, x0_p) -> State:
    """ADMM start from an image (as for the new scheme), with one LM damping per basis."""
    st = state_from_image(prob, x0_c, x0_p)
    st.mu_x = np.full(2, prob.params.lm_mu0)
    return st


def lmcg_iteration(prob: Problem, st: State, m: int = 1, n: int = 1) -> State:
    """One ADMM iteration of LM(m) x CG(n): Eq. 7 (x_c), Eq. 8 (x_p), Eq. 9-11, rho."""
    P = prob.params
    mu_x = np.array(st.mu_x, dtype=np.float64)
    st = st.copy()
    st.mu_x = mu_x
    y_old, z_old = st.y.copy(), st.z.copy()
    for b in (0, 1):
        for _ in range(m):
            lm_step(prob, st, b, n)

    # Eq. 9-10
    Dx = np.stack([grad(st.x[b]) for b in (0, 1)])
    st.y = np.stack([shrinkage(Dx[b] - st.uy[b], P.lam[b] / st.rho[b]) for b in (0, 1)])
    st.z = np.maximum(0.0, st.x - st.uz)
    # Eq. 11 (no a-block in this scheme)
    st.uy = st.uy + st.y - Dx
    st.uz = st.uz + st.z - st.x

    residual_balance(st, P, None, y_old, z_old, Dx, a_block=False)
    st.a = st.Rx.copy()
    st.iteration += 1
    return st
