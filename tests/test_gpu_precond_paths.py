"""The preconditioner's FFT paths at the ends of their range (Sec. 3.3, Eq. 12).

A padded axis of length 64..2048 runs as two half-length register FFTs per warp pair; the other
lengths (32 and 4096) take shared-memory stages, and the column pass maps a stored column to its
frequency when the rows were split. Three parallel-beam slices reach every combination: 12 x 12
(32 x 32: both axes staged), 1040 x 40 (rows of 4096 staged, columns of 128 split) and 40 x 1040 (rows
of 128 split, columns of 4096 staged, reading the split rows' column order). Each matches the FP64
oracle after three ADMM iterations from the oracle's starting image (relative L2 <= 1e-4 in both
bases, 100 keV PE reference), and the three solved as one batch equal their single-slice solves bit
for bit (the path depends on the slice alone)."""
import math

import numpy as np
import pytest

from conftest import rel_l2, to_dev
from oracle import admm as oadmm
from synth import geometry as G
from synth.workloads import baggage_phantom, make_case

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4


def _r32(a):
    return np.float32(a).astype(np.float64)


def _cases():
    geoms = [G.Geometry(G.PARALLEL, 12, 12, 0.5, 30, 0.0, math.pi, 24, 0.5),
             G.Geometry(G.PARALLEL, 1040, 40, 0.05, 48, 0.0, math.pi, 1100, 0.05),
             G.Geometry(G.PARALLEL, 40, 1040, 0.05, 48, 0.0, math.pi, 1100, 0.05)]
    out = []
    for k, g in enumerate(geoms):
        c = make_case(g, lambda gg, r: baggage_phantom(gg, r, n_objects=6), 1e5, 300 + k, e_ref_kev=100.0)
        for key in ("m_h", "m_l", "w_h", "w_l"):
            c[key] = _r32(c[key])
        out.append(c)
    return out


@pytest.fixture(scope="module")
def cases():
    return _cases()


def _start(c):
    prob = oadmm.Problem(c["geom"], c["spectra"], c["m_h"], c["m_l"], c["w_h"], c["w_l"], oadmm.Params())
    return prob, _r32(np.stack(oadmm.initial_image(prob)))


def _solver(cs, dev, x0s):
    from paper_1905_00934_gb300 import Geometry, Solver, Spectra

    geos = [Geometry(c["geom"]) for c in cs]
    sol = Solver(geos, Spectra.from_tables(cs[0]["spectra"]), bp_view_groups=4)
    for b, c in enumerate(cs):
        sol.set_data(b, *[to_dev(c[k], dev) for k in ("m_h", "m_l", "w_h", "w_l")], to_dev(x0s[b], dev))
    sol._keep = geos
    return sol


@pytest.mark.parametrize("which", [0, 1, 2], ids=["32x32", "4096x128", "128x4096"])
def test_precond_paths_match_oracle(cuda_dev, cases, which):
    from paper_1905_00934_gb300 import dect

    c = cases[which]
    prob, x0 = _start(c)
    st = oadmm.state_from_image(prob, x0[0], x0[1])
    for _ in range(3):
        st = oadmm.admm_iteration(prob, st)
    sol = _solver([c], cuda_dev, [x0])
    sol.step(3)
    x = sol.get(0, dect.X).cpu().numpy()
    e_c, e_p = rel_l2(x[0], st.x[0]), rel_l2(x[1], st.x[1])
    print(f"{c['geom'].nx} x {c['geom'].ny}: Compton rel-L2 {e_c:.2e}, PE rel-L2 {e_p:.2e}")
    assert e_c <= IMG_TOL and e_p <= IMG_TOL


def test_mixed_precond_paths_in_one_batch_equal_single_slices(cuda_dev, cases):
    from paper_1905_00934_gb300 import dect

    x0s = [_start(c)[1] for c in cases]
    batch = _solver(cases, cuda_dev, x0s)
    batch.step(3)
    for b, c in enumerate(cases):
        one = _solver([c], cuda_dev, [x0s[b]])
        one.step(3)
        assert np.array_equal(batch.get(b, dect.X).cpu().numpy(), one.get(0, dect.X).cpu().numpy()), b
