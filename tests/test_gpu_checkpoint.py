"""Checkpoint and resume of the batched solver (dect_admm_state_bytes / dect_admm_save /
dect_admm_load): a solver restored from a state image continues bit for bit as the saved one
would have, for both splittings; images of other solvers are rejected without touching the state."""
import math

import numpy as np
import pytest
import torch

from conftest import to_dev
from synth import geometry as G
from synth.workloads import baggage_phantom, make_case, small_parallel_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cases():
    small = small_parallel_case(e_ref_kev=100.0)
    g = G.Geometry(G.FAN_FLAT, 70, 58, 0.12, 90, 0.3, 2 * math.pi, 130, 0.15, 0.02, 16.0, 27.0)
    fan = make_case(g, lambda gg, r: baggage_phantom(gg, r, n_objects=8), 2e5, 91, e_ref_kev=100.0)
    return [small, fan]


def _solver(cases, dev, **params):
    from paper_1905_00934_gb300 import Geometry, Solver, Spectra

    geos = [Geometry(c["geom"]) for c in cases]
    sol = Solver(geos, Spectra.from_tables(cases[0]["spectra"]), bp_view_groups=4, **params)
    for b, c in enumerate(cases):
        sol.set_data(b, *[to_dev(c[k], dev) for k in ("m_h", "m_l", "w_h", "w_l")])
        sol.set_truth(b, to_dev(np.stack([c["truth_c"], c["truth_p"]]), dev))
    sol._keep = geos
    return sol


@pytest.mark.parametrize("scheme", [0, 1])
def test_resume_continues_bit_for_bit(cuda_dev, cases, scheme):
    from paper_1905_00934_gb300 import dect

    a = _solver(cases, cuda_dev, scheme=scheme)
    a.reconstruct(3)
    image = a.save()
    a.step(2)
    b = _solver(cases, cuda_dev, scheme=scheme)
    b.load(image)
    b.step(2)
    for k in range(len(cases)):
        for which in (dect.X, dect.Y, dect.Z, dect.UZ):
            assert torch.equal(a.get(k, which), b.get(k, which))
        sa, sb = a.stats(k), b.stats(k)
        for key in ("iteration", "rho", "r_pri", "r_dual", "xi_db", "count_R", "count_RT", "count_f"):
            assert sa[key] == sb[key], key


def test_load_rejects_images_of_other_solvers(cuda_dev, cases):
    from paper_1905_00934_gb300 import dect

    a = _solver(cases, cuda_dev)
    a.reconstruct(1)
    image = a.save()
    x = a.get(0, dect.X).clone()
    others = [_solver(cases[:1], cuda_dev),                   # another number of slices
              _solver(cases[::-1], cuda_dev),                 # the same slices in another order
              _solver(cases, cuda_dev, scheme=dect.SCHEME_LM_CG),
              _solver(cases, cuda_dev, storage=dect.STORE_F16),
              _solver(cases, cuda_dev, lambda_c=2e-5),         # another TV weight
              _solver(cases, cuda_dev, precondition=dect.PRECOND_RAMP),
              _solver(cases, cuda_dev, udm_f64=1)]
    for o in others:
        with pytest.raises(dect.DectError) as e:
            o.load(image)
        assert e.value.status == dect.EINVAL
    bad = image.copy()
    bad[0] ^= 0xFF
    for img in (image[:-1], bad):
        with pytest.raises(dect.DectError) as e:
            a.load(img)
        assert e.value.status == dect.EINVAL
    # the rejected loads left the state alone; reloading its own image restores the same state
    assert torch.equal(a.get(0, dect.X), x)
    a.load(image)
    assert torch.equal(a.get(0, dect.X), x)
