"""Pins for the oracle's comparison scheme LM(m) x CG(n) (Eq. 6-11 with Eq. 7-8 solved by LM + CG)."""
import numpy as np
import pytest

from oracle import admm, lmcg, projector
from synth import geometry as G
from synth import spectra


class _Mono:
    """Two monochromatic spectra: f is linear, f_k = f_KN(E_k) a_c + f_p(E_k) a_p."""

    def __init__(self):
        e = np.array([50.0, 90.0])
        self.energy_kev = e
        self.s_high = np.array([0.0, 1.0])
        self.s_low = np.array([1.0, 0.0])
        self.f_kn = spectra.klein_nishina(e)
        self.f_p = spectra.photoelectric(e, 60.0)


def _phantom(n=16):
    yy, xx = np.mgrid[0:n, 0:n] - (n - 1) / 2
    xc = 0.2 + 0.1 * ((xx / 6) ** 2 + (yy / 5) ** 2 < 1)
    xp = 0.05 + 0.05 * ((xx + 2) ** 2 + (yy - 1) ** 2 < 9)
    return xc, xp


def _mono_problem(lam=(0.0, 0.0), rho0=(0.1, 0.1), noise=0.0, seed=0):
    g = G.parallel_geometry(16, 30, 24, 1.0, 1.0)
    s = _Mono()
    xc, xp = _phantom()
    Rc, Rp = projector.project(g, xc), projector.project(g, xp)
    rng = np.random.default_rng(seed)
    m_h = s.f_kn[1] * Rc + s.f_p[1] * Rp + noise * rng.normal(size=Rc.shape)
    m_l = s.f_kn[0] * Rc + s.f_p[0] * Rp + noise * rng.normal(size=Rc.shape)
    P = admm.Params(lam=lam, rho0=rho0, m_udm=2, n_pcg=4, precondition=False)
    w = np.full_like(m_h, 3.0)
    return admm.Problem(g, s, m_h, m_l, w, 2 * w, P), xc, xp


def _dense_D(ny, nx):
    n = ny * nx
    Dm = np.zeros((2 * n, n))
    for j in range(ny):
        for i in range(nx):
            p = j * nx + i
            if i < nx - 1:
                Dm[p, p], Dm[p, p + 1] = -1.0, 1.0
            if j < ny - 1:
                Dm[n + p, p], Dm[n + p, p + nx] = -1.0, 1.0
    return Dm


@pytest.mark.parametrize("b", [0, 1])
def test_lm_step_reaches_the_dense_minimiser_of_the_linear_subproblem(b):
    # linear f: the x_b subproblem of Eq. 7 / 8 is quadratic, so one Gauss-Newton step with the
    # linear system solved to convergence and (almost) no damping is its exact minimiser
    prob, xc, xp = _mono_problem()
    g = prob.geom
    rng = np.random.default_rng(1)
    st = lmcg.lmcg_state(prob, 0.5 * xc + 0.05, 0.5 * xp + 0.01)
    st.y = st.y + 0.01 * rng.normal(size=st.y.shape)
    st.uy = 0.01 * rng.normal(size=st.uy.shape)
    st.z = st.z + 0.01 * rng.normal(size=st.z.shape)
    st.uz = 0.01 * rng.normal(size=st.uz.shape)
    st.rho = np.array([0.3, 0.7])
    st.mu_x = np.array([1e-10, 1e-10])
    other = 1 - b
    assert lmcg.lm_step(prob, st, b, 400)

    s = prob.spec
    kh, kl = (s.f_kn[1], s.f_kn[0]) if b == 0 else (s.f_p[1], s.f_p[0])
    oh, ol = (s.f_p[1], s.f_p[0]) if b == 0 else (s.f_kn[1], s.f_kn[0])
    R = projector.matrix(g)
    Dm = _dense_D(g.ny, g.nx)
    wh, wl = prob.w_h.ravel(), prob.w_l.ravel()
    Ro = R @ st.x[other].ravel()
    rho = st.rho[b]
    t = (st.y[b] + st.uy[b]).reshape(2, -1).ravel()
    sz = (st.z[b] + st.uz[b]).ravel()
    A = R.T @ ((wh * kh * kh + wl * kl * kl)[:, None] * R) + rho * (Dm.T @ Dm + np.eye(g.n_pixels))
    rhs = R.T @ (wh * kh * (prob.m_h.ravel() - oh * Ro) + wl * kl * (prob.m_l.ravel() - ol * Ro)) \
        + rho * (Dm.T @ t + sz)
    x_star = np.linalg.solve(A, rhs)
    assert np.linalg.norm(st.x[b].ravel() - x_star) <= 1e-8 * np.linalg.norm(x_star)
    # R x is carried consistently
    assert np.allclose(st.Rx[b].ravel(), R @ st.x[b].ravel(), rtol=1e-10, atol=1e-12)


def test_lm_never_increases_the_subproblem_objective_and_damping_moves_by_ten():
    from synth.workloads import small_parallel_case

    c = small_parallel_case(e_ref_kev=100.0)
    prob = admm.Problem(c["geom"], c["spectra"], c["m_h"], c["m_l"], c["w_h"], c["w_l"], admm.Params())
    xc0, xp0 = admm.initial_image(prob)
    st = lmcg.lmcg_state(prob, xc0, xp0)

    def objective(b):
        rh, rl = lmcg._data_terms(prob, st.Rx, False)
        return lmcg._data_cost(prob, rh, rl) + lmcg._al_cost(st.rho[b], st.x[b], st.y[b] + st.uy[b],
                                                               st.z[b] + st.uz[b])

    for b in (0, 1, 0, 1):
        for _ in range(3):
            before, mu = objective(b), st.mu_x[b]
            acc = lmcg.lm_step(prob, st, b, 2)
            after = objective(b)
            assert after <= before
            assert st.mu_x[b] == pytest.approx(mu * (0.1 if acc else 10.0))
            assert acc == (after < before)


@pytest.mark.parametrize("m,n", [(1, 1), (2, 3)])
def test_table1_operation_counts(m, n):
    prob, xc, xp = _mono_problem()
    st = lmcg.lmcg_state(prob, xc, xp)
    before = (prob.count.R, prob.count.RT, prob.count.f)
    for _ in range(3):
        st = lmcg.lmcg_iteration(prob, st, m, n)
    assert prob.count.R - before[0] == 3 * 2 * m * (n + 1)
    assert prob.count.RT - before[1] == 3 * 2 * m * (n + 1)
    assert prob.count.f - before[2] == 3 * 4 * m


def test_truth_is_a_fixed_point_noise_free():
    # exact linear data, lambda = 0: at the phantom the gradient vanishes, so no step is accepted
    # and y, z, u, x stay put
    prob, xc, xp = _mono_problem()
    st0 = lmcg.lmcg_state(prob, xc, xp)
    st = lmcg.lmcg_iteration(prob, st0, 2, 5)
    assert np.allclose(st.x, st0.x, atol=1e-12)
    assert np.allclose(st.uy, 0.0, atol=1e-12) and np.allclose(st.uz, 0.0, atol=1e-12)


def test_both_schemes_converge_to_the_same_map_point():
    # the two splittings solve the same problem (Eq. 4): with noisy data and TV the MAP point is not
    # the phantom, and both ADMM schemes approach it (to within a small fraction of their distance
    # from the start)
    prob, xc, xp = _mono_problem(lam=(2e-2, 2e-2), rho0=(0.5, 0.5), noise=0.02, seed=3)
    prob.params.adapt_rho = False
    start = (np.full((16, 16), 0.15), np.full((16, 16), 0.06))
    st_l = lmcg.lmcg_state(prob, *start)
    for _ in range(400):
        st_l = lmcg.lmcg_iteration(prob, st_l, 2, 8)
    st_u = admm.state_from_image(prob, *start)
    for _ in range(400):
        st_u = admm.admm_iteration(prob, st_u)
    x_start = np.stack(start)
    for b in (0, 1):
        d = np.linalg.norm(st_l.x[b] - st_u.x[b])
        assert d <= 2e-3 * np.linalg.norm(st_u.x[b] - x_start[b]), (b, d)
