"""The MAP objective of Eq. 4 as a GPU monitor (dect_params.objective_every).

The solver evaluates 1/2 ||f(R x) - m||^2_Sigma + sum_b lambda_b ||D x_b||_1 at its current images
after every k-th iteration. Each check evaluates the oracle's objective (oracle.admm.map_objective:
a float64 projection, the float64 forward model) at the GPU's own images, so only the objective's
arithmetic is compared: relative difference <= 1e-6 on the small parallel workload (float64 and
float32 storage) and on a 128^2 fan slice. Turning the monitor on changes neither the iterates nor
Table 1's operation counts."""
import math

import numpy as np
import pytest
import torch

from conftest import to_dev
from oracle import admm as oadmm
from synth import geometry as G
from synth.workloads import baggage_phantom, make_case, small_parallel_case

pytestmark = pytest.mark.gpu

TOL = 1e-6


def _r32(a):
    return np.float32(a).astype(np.float64)


def _fan128():
    g = G.Geometry(G.FAN_FLAT, 128, 128, 0.4, 180, 0.0, 2 * math.pi, 256, 0.7, 0.0, 55.0, 95.0)
    return make_case(g, lambda gg, r: baggage_phantom(gg, r, n_objects=10), 2e5, 77, e_ref_kev=100.0)


@pytest.fixture(scope="module")
def cases():
    out = {"small_literal": small_parallel_case(e_ref_kev=1.0), "small_100": small_parallel_case(e_ref_kev=100.0),
           "fan128": _fan128()}
    for c in out.values():
        for k in ("m_h", "m_l", "w_h", "w_l"):
            c[k] = _r32(c[k])
    return out


def _run(c, dev, iters, **params):
    from paper_1905_00934_gb300 import Geometry, Solver, Spectra, dect

    geo = Geometry(c["geom"])
    sol = Solver([geo], Spectra.from_tables(c["spectra"]), **params)
    sol.set_data(0, *[to_dev(c[k], dev) for k in ("m_h", "m_l", "w_h", "w_l")])
    sol._keep = geo
    sol.reconstruct(iters)
    return sol, sol.stats(0), sol.get(0, dect.X).cpu().double().numpy()


@pytest.mark.parametrize("name,storage", [("small_literal", 3), ("small_100", 0), ("fan128", 0)],
                         ids=["small_literal_f64", "small_100_f32", "fan128_f32"])
def test_objective_matches_oracle_at_the_same_images(cuda_dev, cases, name, storage):
    c = cases[name]
    sol, st, x = _run(c, cuda_dev, 6, storage=storage, objective_every=3)
    assert st["objective_iteration"] == 6
    prob = oadmm.Problem(c["geom"], c["spectra"], c["m_h"], c["m_l"], c["w_h"], c["w_l"], oadmm.Params())
    ref = oadmm.map_objective(prob, x)
    rel = abs(st["objective"] - ref) / abs(ref)
    print(f"{name}, storage {storage}: objective {st['objective']:.10e}, oracle at the same x {ref:.10e}, rel {rel:.2e}")
    assert rel <= TOL


def test_objective_monitor_changes_nothing_else(cuda_dev, cases):
    c = cases["small_100"]
    # two solvers: the backprojector's view-group count (the order of its partial sums) fixed for both
    a, sa, xa = _run(c, cuda_dev, 7, objective_every=2, bp_view_groups=4)
    b, sb, xb = _run(c, cuda_dev, 7, bp_view_groups=4)
    assert np.array_equal(xa, xb)
    assert (sa["count_R"], sa["count_RT"], sa["count_f"]) == (sb["count_R"], sb["count_RT"], sb["count_f"])
    assert sa["objective_iteration"] == 6 and math.isnan(sb["objective"]) and sb["objective_iteration"] == -1
