"""Pins for the oracle's ADMM pieces: D, shrinkage, preconditioner, PCG (Eq. 12), the
iteration (Eq. 9-13), its operation counts (Table 1) and its convergence."""

import numpy as np
import pytest

from oracle import admm, projector
from synth import geometry as G
from synth import spectra


def _dense_D(ny, nx):
    """D as an explicit matrix from the forward-difference definition."""
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


def test_grad_and_adjoint_against_explicit_matrix():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(5, 7))
    y = rng.normal(size=(2, 5, 7))
    Dm = _dense_D(5, 7)
    assert np.allclose(admm.grad(x).ravel(), Dm @ x.ravel())
    assert np.allclose(admm.grad_t(y).ravel(), Dm.T @ y.ravel())
    assert np.allclose(admm.grad(np.full((4, 4), 3.0)), 0.0)


def test_shrinkage_closed_form():
    t = np.array([-3.0, -1.0, -0.5, 0.0, 0.2, 1.0, 2.5])
    assert np.allclose(admm.shrinkage(t, 1.0), [-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.5])
    assert np.allclose(admm.shrinkage(t, 0.0), t)
    # it is the proximal map of tau*|.|: minimises tau|y| + (y - t)^2 / 2 over a fine grid
    grid = np.linspace(-4, 4, 80001)
    for ti in t:
        yb = grid[np.argmin(1.0 * np.abs(grid) + 0.5 * (grid - ti) ** 2)]
        assert admm.shrinkage(np.array([ti]), 1.0)[0] == pytest.approx(yb, abs=1e-4)


def test_xi_metric():
    x = np.ones(10)
    assert admm.xi_db(1.1 * x, x) == pytest.approx(-20.0)
    assert admm.xi_db(2.0 * x, x) == pytest.approx(0.0)


def test_pad_size():
    assert [admm.pad_size(n) for n in (8, 64, 96, 512, 1000)] == [16, 128, 256, 1024, 2048]


def test_preconditioner_symmetric_positive_definite():
    g = G.parallel_geometry(12, 20, 18, 0.1, 0.1)
    H = admm.precond_response(g)
    assert np.all(H > 0) and np.all(H <= 1.0)
    # even in frequency: H(k) = H(-k), so M^-1 is a real symmetric operator
    assert np.allclose(H, np.roll(H[::-1, ::-1], 1, axis=(0, 1)))
    n = 144
    M = np.stack([admm.apply_precond(H, e.reshape(12, 12)).ravel() for e in np.eye(n)], axis=1)
    assert np.allclose(M, M.T, atol=1e-12)
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_preconditioner_models_the_operator_at_low_frequency():
    # for a shift-invariant model (image centre), M^-1 A applied to a smooth centred bump is close to it
    g = G.parallel_geometry(48, 96, 72, 0.1, 0.1)
    H = admm.precond_response(g)
    yy, xx = np.mgrid[0:48, 0:48] - 23.5
    bump = np.exp(-(xx**2 + yy**2) / (2 * 4.0**2))
    A = projector.backproject(g, projector.project(g, bump)) + admm.grad_t(admm.grad(bump)) + bump
    ratio = np.vdot(admm.apply_precond(H, A), bump) / np.vdot(bump, bump)
    assert 0.9 < ratio < 1.1
    # without preconditioning the same ratio is the operator's size, orders of magnitude off
    assert np.vdot(A, bump) / np.vdot(bump, bump) > 10


def _eq12_dense(g):
    Rm = projector.matrix(g)
    Dm = _dense_D(g.ny, g.nx)
    return Rm, Dm, Rm.T @ Rm + Dm.T @ Dm + np.eye(g.n_pixels)


@pytest.mark.parametrize("precondition", [admm.PRECOND_NONE, admm.PRECOND_CIRCULANT, admm.PRECOND_RAMP])
def test_pcg_converges_to_dense_cholesky_solution(precondition):
    g = G.parallel_geometry(8, 9, 12, 0.1, 0.1, angle0_rad=0.05)
    Rm, Dm, A = _eq12_dense(g)
    rng = np.random.default_rng(1)
    P = admm.Params(precondition=precondition)
    t = spectra.SpectralTables()
    prob = admm.Problem(g, t, np.zeros((9, 12)), np.zeros((9, 12)), np.ones((9, 12)), np.ones((9, 12)), P)
    st = admm.state_from_image(prob, rng.normal(size=(8, 8)), rng.normal(size=(8, 8)))
    st.a = rng.normal(size=st.a.shape)
    st.ua = rng.normal(size=st.ua.shape)
    st.y = rng.normal(size=st.y.shape)
    st.uy = rng.normal(size=st.uy.shape)
    st.z = rng.normal(size=st.z.shape)
    st.uz = rng.normal(size=st.uz.shape)
    admm.pcg_x_update(prob, st, 64, True, prob.H)
    L = np.linalg.cholesky(A)
    for b in (0, 1):
        rhs = Rm.T @ (st.a[b] + st.ua[b]).ravel() + Dm.T @ (st.y[b] + st.uy[b]).ravel() + (st.z[b] + st.uz[b]).ravel()
        sol = np.linalg.solve(L.T, np.linalg.solve(L, rhs))
        assert np.allclose(st.x[b].ravel(), sol, rtol=1e-10, atol=1e-10)
        # the carried R x equals R applied to the final x
        assert np.allclose(st.Rx[b].ravel(), Rm @ st.x[b].ravel(), atol=1e-10)


def test_preconditioner_speeds_up_cg():
    g = G.parallel_geometry(32, 48, 48, 0.1, 0.1)
    rng = np.random.default_rng(2)
    errs = {}
    for pc in (False, True):
        P = admm.Params(precondition=pc)
        t = spectra.SpectralTables()
        prob = admm.Problem(g, t, np.zeros((48, 48)), np.zeros((48, 48)), np.ones((48, 48)), np.ones((48, 48)), P)
        st = admm.state_from_image(prob, np.zeros((32, 32)), np.zeros((32, 32)))
        st.a = np.stack([projector.project(g, rng.uniform(size=(32, 32)))] * 2)
        ref = st.copy()
        admm.pcg_x_update(prob, ref, 300, True, prob.H)
        admm.pcg_x_update(prob, st, 8, True, prob.H)
        errs[pc] = np.linalg.norm(st.x - ref.x) / np.linalg.norm(ref.x)
    assert errs[True] < 0.5 * errs[False]


@pytest.mark.parametrize("m,n", [(1, 1), (2, 3), (3, 1)])
def test_table1_operation_counts(m, n):
    # UDM(m)-PCG(n): R 2n, R^T 2(n+1), f 4m per ADMM iteration (both bases)
    g = G.parallel_geometry(16, 12, 24, 0.1, 0.1)
    t = spectra.SpectralTables()
    rng = np.random.default_rng(3)
    m_h = rng.uniform(0.1, 1.0, (12, 24))
    P = admm.Params(m_udm=m, n_pcg=n)
    prob = admm.Problem(g, t, m_h, m_h * 1.1, np.full((12, 24), 1e4), np.full((12, 24), 1e4), P)
    st = admm.state_from_image(prob, np.full((16, 16), 0.1), np.full((16, 16), 1e-3))
    before = (prob.count.R, prob.count.RT, prob.count.f)
    for _ in range(3):
        st = admm.admm_iteration(prob, st)
    assert prob.count.R - before[0] == 3 * 2 * n
    assert prob.count.RT - before[1] == 3 * 2 * (n + 1)
    assert prob.count.f - before[2] == 3 * 4 * m


class _Mono:
    def __init__(self):
        e = np.array([50.0, 90.0])
        self.energy_kev = e
        self.s_high = np.array([0.0, 1.0])
        self.s_low = np.array([1.0, 0.0])
        self.f_kn = spectra.klein_nishina(e)
        self.f_p = spectra.photoelectric(e, 60.0)


def _mono_problem(lam=(0.0, 0.0), rho0=(0.1, 0.1)):
    g = G.parallel_geometry(16, 30, 24, 1.0, 1.0)
    s = _Mono()
    yy, xx = np.mgrid[0:16, 0:16] - 7.5
    xc = 0.2 + 0.1 * ((xx / 6) ** 2 + (yy / 5) ** 2 < 1)
    xp = 0.05 + 0.05 * ((xx + 2) ** 2 + (yy - 1) ** 2 < 9)
    Rc, Rp = projector.project(g, xc), projector.project(g, xp)
    m_h = s.f_kn[1] * Rc + s.f_p[1] * Rp
    m_l = s.f_kn[0] * Rc + s.f_p[0] * Rp
    P = admm.Params(lam=lam, rho0=rho0, m_udm=2, n_pcg=4)
    return admm.Problem(g, s, m_h, m_l, np.ones_like(m_h), np.ones_like(m_h), P), xc, xp


def test_admm_truth_is_a_fixed_point_noise_free_monochromatic():
    # exact data, lambda = 0: starting at the phantom with zero duals, an iteration changes nothing
    prob, xc, xp = _mono_problem()
    st0 = admm.state_from_image(prob, xc, xp)
    st = admm.admm_iteration(prob, st0)
    assert np.allclose(st.x, st0.x, atol=1e-12)
    assert np.allclose(st.a, st0.a, atol=1e-12)
    assert np.allclose(st.ua, 0.0, atol=1e-12) and np.allclose(st.uy, 0.0, atol=1e-12)
    assert np.allclose(st.uz, 0.0, atol=1e-12)


def test_admm_converges_to_exact_solution_noise_free_monochromatic():
    # noise-free, linear f, lambda = 0, positive truth: the MAP point is the phantom itself;
    # ADMM drives x towards it and both residuals towards zero
    prob, xc, xp = _mono_problem()
    st = admm.state_from_image(prob, np.full((16, 16), 0.1), np.full((16, 16), 0.05))
    err0 = (np.linalg.norm(st.x[0] - xc) / np.linalg.norm(xc), np.linalg.norm(st.x[1] - xp) / np.linalg.norm(xp))
    first = None
    for it in range(300):
        st = admm.admm_iteration(prob, st)
        if first is None:
            first = (st.r_pri.copy(), st.r_dual.copy())
    err_c = np.linalg.norm(st.x[0] - xc) / np.linalg.norm(xc)
    err_p = np.linalg.norm(st.x[1] - xp) / np.linalg.norm(xp)
    assert err_c < 1e-2 * err0[0] * 10 and err_c < 5e-3 and err_p < 1e-2
    assert np.all(st.r_pri < 1e-2 * first[0]) and np.all(st.r_dual < 1e-1 * first[1])


def test_small_case_objective_and_residuals_trend():
    # the small parallel-beam workload: MAP objective (Eq. 4) falls well below its start and
    # the primal residual of both bases shrinks over 20 iterations
    from synth.workloads import small_parallel_case
    c = small_parallel_case()
    prob = admm.Problem(c["geom"], c["spectra"], c["m_h"], c["m_l"], c["w_h"], c["w_l"], admm.Params())
    xc0, xp0 = admm.initial_image(prob)
    st = admm.state_from_image(prob, xc0, xp0)
    obj0 = admm.map_objective(prob, st.x)
    st = admm.admm_iteration(prob, st)
    r0 = st.r_pri.copy()
    for _ in range(19):
        st = admm.admm_iteration(prob, st)
    assert admm.map_objective(prob, st.x) < 0.2 * obj0
    assert np.all(st.r_pri < r0)
    # the Compton estimate improves on the initial image over the first iterations
    assert admm.xi_db(st.x[0], c["truth_c"]) < admm.xi_db(xc0, c["truth_c"]) + 3.0


@pytest.mark.parametrize("nx,nv,nb,dx,du", [(48, 96, 72, 0.1, 0.1), (64, 90, 96, 0.1, 0.1),
                                           (40, 60, 64, 0.1, 0.15), (32, 120, 80, 0.05, 0.04)])
def test_point_response_follows_the_continuous_parallel_beam_constant(nx, nv, nb, dx, du):
    # continuous parallel beam, V views over pi, pixel dx, bin pitch du: the backprojection of the
    # projection of a point is (V / pi) (dx^4 / du) / r at distance r (the angular integral of
    # delta(r cos phi) over [0, pi) is 1 / r), whose 2D Fourier transform on the pixel grid is
    # 2 V dx^3 / (du |w|). The discrete point response at w = pi/4 (the ramp constant K) carries
    # that constant up to the Joseph interpolation footprint (a few per cent at pi/4).
    g = G.parallel_geometry(nx, nv, nb, dx, du)
    phat = admm.point_response_dft(g)
    K = phat[0, phat.shape[1] // 8] * np.pi / 4
    assert K == pytest.approx(2 * nv * dx**3 / du, rel=0.12)
    # same constant along y (the operator is isotropic)
    assert phat[phat.shape[0] // 8, 0] == pytest.approx(phat[0, phat.shape[1] // 8], rel=1e-9)


def test_ramp_response_shape():
    g = G.parallel_geometry(32, 120, 80, 0.05, 0.04)
    H = admm.ramp_response(g)
    py, px = H.shape
    assert (py, px) == (64, 64)
    assert np.all(H > 0) and np.all(H < 1)
    # real and even in frequency, and radial: equal wherever |w| is equal
    assert np.allclose(H, np.roll(H[::-1, ::-1], 1, axis=(0, 1)))
    assert np.allclose(H, H.T)
    assert H[3, 4] == pytest.approx(H[0, 5]) and H[60, 3] == pytest.approx(H[5, 0])
    # increasing with |w| along the axis up to Nyquist; DC takes the first non-zero frequency
    assert np.all(np.diff(H[0, 1 : px // 2 + 1]) > 0)
    assert H[0, 0] == H[0, 1]
    # at the calibration frequency (0, pi/4) it equals the circulant model without D^T D
    phat = admm.point_response_dft(g)
    assert H[0, px // 8] == pytest.approx(1.0 / (phat[0, px // 8] + 1.0), rel=1e-12)
    assert H[0, px // 8] == pytest.approx(admm.precond_response(g, False)[0, px // 8], rel=1e-12)
    # H = |w| / (K + |w|) at a diagonal frequency, with |w| written out
    K = phat[0, px // 8] * np.pi / 4
    w = np.hypot(2 * np.pi * 5 / py, 2 * np.pi * 7 / px)
    assert H[5, px - 7] == pytest.approx(w / (K + w), rel=1e-12)


def test_ramp_preconditioner_ranks_between_none_and_circulant():
    # R^T R-dominated operator (many views): the plain ramp speeds CG up over no preconditioner,
    # the full circulant model (which also carries D^T D) more
    g = G.parallel_geometry(32, 360, 48, 0.1, 0.1)
    rng = np.random.default_rng(2)
    xt = rng.uniform(size=(32, 32))
    errs = {}
    for pc in (admm.PRECOND_NONE, admm.PRECOND_CIRCULANT, admm.PRECOND_RAMP):
        P = admm.Params(precondition=pc)
        z = np.zeros((360, 48))
        prob = admm.Problem(g, spectra.SpectralTables(), z, z, z + 1, z + 1, P)
        st = admm.state_from_image(prob, np.zeros((32, 32)), np.zeros((32, 32)))
        st.a = np.stack([projector.project(g, xt)] * 2)
        ref = st.copy()
        admm.pcg_x_update(prob, ref, 400, True, prob.H)
        admm.pcg_x_update(prob, st, 8, True, prob.H)
        errs[pc] = np.linalg.norm(st.x - ref.x) / np.linalg.norm(ref.x)
    assert errs[admm.PRECOND_CIRCULANT] < 0.1 * errs[admm.PRECOND_RAMP]
    assert errs[admm.PRECOND_RAMP] < 0.2 * errs[admm.PRECOND_NONE]


def test_precondition_mode_is_validated():
    g = G.parallel_geometry(8, 9, 12, 0.1, 0.1)
    z = np.zeros((9, 12))
    with pytest.raises(ValueError):
        admm.Problem(g, spectra.SpectralTables(), z, z, z + 1, z + 1, admm.Params(precondition=3))


# ---- residual balancing (Sec. 3.2, Boyd et al. Sec. 3.4.1): the rho rule and the dual rescale ----

def _balance_state(rho):
    """A hand-made state after the dual update: one non-zero entry per block, so that per basis
    ||a - R x||, ||y - D x||, ||z - x|| = 6, 2, 3 (r_pri = 7) and ||a - a_old||, ||y - y_old||,
    ||z - z_old|| = 2, 1, 2 (r_dual = 3 rho); every scaled dual entry is 1 + its index."""
    V, Nb, ny, nx = 1, 3, 2, 2
    z4 = lambda *s: np.zeros(s)
    st = admm.State(x=z4(2, ny, nx), Rx=z4(2, V, Nb), a=z4(2, V, Nb), ua=z4(2, V, Nb), y=z4(2, 2, ny, nx),
                    uy=z4(2, 2, ny, nx), z=z4(2, ny, nx), uz=z4(2, ny, nx), rho=np.array(rho, dtype=np.float64),
                    mu=z4(V, Nb), status=np.zeros((V, Nb), np.uint8))
    for u in (st.ua, st.uy, st.uz):
        u[...] = 1.0 + np.arange(u.size).reshape(u.shape)
    Dx = z4(2, 2, ny, nx)
    a_old, y_old, z_old = z4(2, V, Nb), z4(2, 2, ny, nx), z4(2, ny, nx)
    for b in (0, 1):
        st.a[b, 0, 1] = 6.0           # a - R x
        a_old[b, 0, 1] = 4.0          # a - a_old = 2
        st.y[b, 1, 0, 1] = 2.0        # y - D x (D x = 0)
        y_old[b, 1, 0, 1] = 1.0       # y - y_old = 1
        st.z[b, 1, 1] = 3.0           # z - x (x = 0)
        z_old[b, 1, 1] = 1.0          # z - z_old = 2
    return st, a_old, y_old, z_old, Dx


@pytest.mark.parametrize("rho,expect", [
    ((0.2, 25.0), (2.0, 0.5)),    # r_pri 7 > 10 * 0.6: grow; r_dual 75 > 10 * 7: shrink
    ((20.0, 1.0), (1.0, 1.0)),    # 60 and 3 against 7: neither rule fires
])
def test_residual_balance_rule_and_dual_rescale(rho, expect):
    P = admm.Params(mu_b=10.0, tau=2.0)
    st, a_old, y_old, z_old, Dx = _balance_state(rho)
    before = st.copy()
    admm.residual_balance(st, P, a_old, y_old, z_old, Dx)
    for b in (0, 1):
        # residuals by hand: sqrt(6^2 + 2^2 + 3^2) and rho sqrt(2^2 + 1^2 + 2^2)
        assert st.r_pri[b] == pytest.approx(7.0, rel=1e-15)
        assert st.r_dual[b] == pytest.approx(3.0 * rho[b], rel=1e-15)
        f = expect[b]
        assert st.rho[b] == rho[b] * f
        # scaled duals divided by the factor rho was multiplied by (exact: f is a power of two)
        for name in ("ua", "uy", "uz"):
            assert np.array_equal(getattr(st, name)[b], getattr(before, name)[b] / f), (name, b)
        # the primal blocks are untouched
        for name in ("x", "a", "Rx", "y", "z"):
            assert np.array_equal(getattr(st, name)[b], getattr(before, name)[b])


def test_residual_balance_counts_the_a_block():
    """Without the a-block the same state balances differently: rho 0.2 would stay (r_pri sqrt(13)
    < 10 * 0.2 sqrt(5)) and rho 20 would shrink (20 sqrt(5) > 10 sqrt(13)). With it, 0.2 grows and
    20 stays, and u^a is rescaled only when the a-block takes part."""
    P = admm.Params(mu_b=10.0, tau=2.0)
    st, a_old, y_old, z_old, Dx = _balance_state((0.2, 20.0))
    admm.residual_balance(st, P, a_old, y_old, z_old, Dx)
    assert list(st.rho) == [0.4, 20.0]
    st, a_old, y_old, z_old, Dx = _balance_state((0.2, 20.0))
    ua = st.ua.copy()
    admm.residual_balance(st, P, None, y_old, z_old, Dx, a_block=False)
    assert list(st.rho) == [0.2, 10.0]
    assert st.r_pri[0] == pytest.approx(np.sqrt(13.0), rel=1e-15)
    assert st.r_dual[1] == pytest.approx(20.0 * np.sqrt(5.0), rel=1e-15)
    assert np.array_equal(st.ua, ua)
    assert np.array_equal(st.uy[1], _balance_state((0.2, 20.0))[0].uy[1] * 2.0)


def test_residual_balance_off_keeps_rho():
    P = admm.Params(mu_b=10.0, tau=2.0, adapt_rho=False)
    st, a_old, y_old, z_old, Dx = _balance_state((0.2, 25.0))
    before = st.copy()
    admm.residual_balance(st, P, a_old, y_old, z_old, Dx)
    assert np.array_equal(st.rho, before.rho) and np.array_equal(st.ua, before.ua)
    assert st.r_pri[0] == pytest.approx(7.0, rel=1e-15)
