"""GPU comparison scheme LM(m) x CG(n) (Sec. 3.2, Eq. 6-11; Table 1) against the FP64 oracle.

Both sides get the same float32-rounded measurements and start from the oracle's initial image.
Each LM step's accept / reject decision is a comparison of the subproblem objective before and
after the trial step over the whole slice; both sides take the same decisions here, and the rho
decisions are equal. Images: relative L2 <= 1e-4 after the iteration count."""
import math

import numpy as np
import pytest

from conftest import rel_l2, to_dev
from oracle import admm as oadmm
from oracle import lmcg as olmcg
from synth import geometry as G
from synth.workloads import baggage_phantom, make_case, small_parallel_case

pytestmark = pytest.mark.gpu


def _r32(a):
    return np.float32(a).astype(np.float64)


def _prepare(c):
    for k in ("m_h", "m_l", "w_h", "w_l"):
        c[k] = _r32(c[k])
    prob = oadmm.Problem(c["geom"], c["spectra"], c["m_h"], c["m_l"], c["w_h"], c["w_l"], oadmm.Params())
    x0 = _r32(np.stack(oadmm.initial_image(prob)))
    return c, x0


@pytest.fixture(scope="module")
def small100():
    return _prepare(small_parallel_case(e_ref_kev=100.0))


@pytest.fixture(scope="module")
def fan_ragged():
    g = G.Geometry(G.FAN_FLAT, 70, 58, 0.12, 90, 0.3, 2 * math.pi, 130, 0.15, 0.02, 16.0, 27.0)
    return _prepare(make_case(g, lambda gg, r: baggage_phantom(gg, r, n_objects=8), 2e5, 91, e_ref_kev=100.0))


def _solver(cases, dev, x0s, **params):
    from paper_1905_00934_gb300 import Geometry, Solver, Spectra, dect

    geos = [Geometry(c["geom"]) for c in cases]
    sol = Solver(geos, Spectra.from_tables(cases[0]["spectra"]), scheme=dect.SCHEME_LM_CG, **params)
    for b, c in enumerate(cases):
        sol.set_data(b, *[to_dev(c[k], dev) for k in ("m_h", "m_l", "w_h", "w_l")],
                     None if x0s[b] is None else to_dev(x0s[b], dev))
        sol.set_truth(b, to_dev(np.stack([c["truth_c"], c["truth_p"]]), dev))
    sol._keep = geos
    return sol


def _run_pair(c, x0, dev, iters, m, n):
    P = oadmm.Params(m_udm=m, n_pcg=n)
    prob = oadmm.Problem(c["geom"], c["spectra"], c["m_h"], c["m_l"], c["w_h"], c["w_l"], P)
    st = olmcg.lmcg_state(prob, x0[0], x0[1])
    sol = _solver([c], dev, [x0], m_udm=m, n_pcg=n)
    hist = []
    for _ in range(iters):
        st = olmcg.lmcg_iteration(prob, st, m, n)
        sol.step(1)
        s = sol.stats(0)
        hist.append((st.rho.copy(), np.array(s["rho"]), st.r_pri.copy(), np.array(s["r_pri"])))
    return st, sol, hist


@pytest.mark.parametrize("m,n,iters", [(1, 1, 10), (2, 3, 5)])
def test_iterations_match_oracle(cuda_dev, small100, m, n, iters):
    from paper_1905_00934_gb300 import dect

    c, x0 = small100
    st, sol, hist = _run_pair(c, x0, cuda_dev, iters, m, n)
    for it, (rho_o, rho_g, rp_o, rp_g) in enumerate(hist):
        assert np.array_equal(rho_o, rho_g), f"rho decision differs at iteration {it + 1}"
        assert np.allclose(rp_g, rp_o, rtol=1e-3)
    x = sol.get(0, dect.X).cpu().numpy()
    e_c, e_p = rel_l2(x[0], st.x[0]), rel_l2(x[1], st.x[1])
    print(f"LM({m}) x CG({n}), {iters} iterations: Compton rel-L2 {e_c:.2e}, PE rel-L2 {e_p:.2e}")
    assert e_c <= 1e-4 and e_p <= 1e-4
    xi = sol.stats(0)["xi_db"]
    assert abs(xi[0] - oadmm.xi_db(st.x[0], c["truth_c"])) < 0.01
    assert abs(xi[1] - oadmm.xi_db(st.x[1], c["truth_p"])) < 0.01


def test_ragged_fan_matches_oracle(cuda_dev, fan_ragged):
    from paper_1905_00934_gb300 import dect

    c, x0 = fan_ragged
    st, sol, _ = _run_pair(c, x0, cuda_dev, 4, 1, 2)
    x = sol.get(0, dect.X).cpu().numpy()
    e_c, e_p = rel_l2(x[0], st.x[0]), rel_l2(x[1], st.x[1])
    print(f"ragged fan, LM(1) x CG(2), 4 iterations: Compton rel-L2 {e_c:.2e}, PE rel-L2 {e_p:.2e}")
    assert e_c <= 1e-4 and e_p <= 1e-4


def test_table1_counts(cuda_dev, small100):
    c, x0 = small100
    for m, n in [(1, 1), (2, 3)]:
        sol = _solver([c], cuda_dev, [x0], m_udm=m, n_pcg=n)
        sol.step(0)
        s0 = sol.stats(0)
        sol.step(3)
        s1 = sol.stats(0)
        # R d is carried through CG, so a step projects n times where Table 1 counts n + 1
        assert s1["count_R"] - s0["count_R"] == 3 * 2 * m * n
        assert s1["count_RT"] - s0["count_RT"] == 3 * 2 * m * (n + 1)
        assert s1["count_f"] - s0["count_f"] == 3 * 4 * m


def test_graph_eager_and_batched_are_bitwise_equal(cuda_dev, small100, fan_ragged):
    from paper_1905_00934_gb300 import dect

    cases = [small100[0], fan_ragged[0]]
    x0s = [small100[1], fan_ragged[1]]
    outs = []
    for use_graph in (1, 0):
        sol = _solver(cases, cuda_dev, x0s, use_graph=use_graph, bp_view_groups=4)
        sol.step(3)
        outs.append([sol.get(b, dect.X).cpu().numpy() for b in range(2)])
    for b in range(2):
        assert np.array_equal(outs[0][b], outs[1][b])
        single = _solver([cases[b]], cuda_dev, [x0s[b]], bp_view_groups=4)
        single.step(3)
        assert np.array_equal(single.get(0, dect.X).cpu().numpy(), outs[0][b])
