"""16-bit storage of the solver's sinogram vectors and projector textures (float32 / float64 arithmetic).

Against the FP64 oracle from the same starting image, after 20 iterations of the small workload with
the photoelectric basis at 100 keV: float32 storage holds 1e-4 (relative L2, both bases); float16 and
bfloat16 storage round every stored line integral to 11 / 8 significant bits, and the errors they
produce are measured and bounded here (Compton and PE reported separately). The full-size subset of
the 1024 x 1024, 1440-view, 2048-bin workload is compared with the oracle's stored values (xi every
10 iterations and sampled pixels after 100 iterations; sampled pixels after the first iterations)
when those references are present."""
import json
import os

import numpy as np
import pytest

from conftest import rel_l2, to_dev
from oracle import admm as oadmm
from synth.workloads import small_parallel_case

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mixed_1024_oracle.json")
GOLDEN_EARLY = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mixed_1024_early.json")


def _r32(a):
    return np.float32(a).astype(np.float64)


@pytest.fixture(scope="module")
def small_ref():
    c = small_parallel_case(e_ref_kev=100.0)
    for k in ("m_h", "m_l", "w_h", "w_l"):
        c[k] = _r32(c[k])
    prob = oadmm.Problem(c["geom"], c["spectra"], c["m_h"], c["m_l"], c["w_h"], c["w_l"], oadmm.Params())
    x0 = _r32(np.stack(oadmm.initial_image(prob)))
    st = oadmm.state_from_image(prob, x0[0], x0[1])
    for _ in range(20):
        st = oadmm.admm_iteration(prob, st)
    return c, x0, st


@pytest.mark.parametrize("storage,bound", [(0, 1e-4), (1, 3e-2), (2, 2e-1)], ids=["f32", "f16", "bf16"])
def test_storage_error_against_oracle(cuda_dev, small_ref, storage, bound):
    from paper_1905_00934_gb300 import Geometry, Solver, Spectra, dect

    c, x0, st = small_ref
    geo = Geometry(c["geom"])
    sol = Solver([geo], Spectra.from_tables(c["spectra"]), storage=storage)
    sol.set_data(0, *[to_dev(c[k], cuda_dev) for k in ("m_h", "m_l", "w_h", "w_l")], to_dev(x0, cuda_dev))
    sol.step(20)
    x = sol.get(0, dect.X).cpu().numpy()
    e_c, e_p = rel_l2(x[0], st.x[0]), rel_l2(x[1], st.x[1])
    print(f"storage {['f32', 'f16', 'bf16'][storage]}: Compton rel-L2 {e_c:.2e}, PE rel-L2 {e_p:.2e}")
    assert e_c <= bound and e_p <= bound


def _mixed_solver(cuda_dev, slices, storage, with_truth):
    from concurrent.futures import ThreadPoolExecutor

    from paper_1905_00934_gb300 import Geometry, Solver, Spectra
    from synth.workloads import BAGGAGE_KAPPA, baggage_fan_case

    with ThreadPoolExecutor(max_workers=len(slices)) as ex:
        cases = list(ex.map(lambda s: baggage_fan_case(slice_index=s["slice_index"], n=1024, n_views=1440,
                                                        n_bins=2048), slices))
    geos = [Geometry(c["geom"]) for c in cases]
    sol = Solver(geos, Spectra.from_tables(cases[0]["spectra"]), kappa=BAGGAGE_KAPPA, storage=storage)
    for b, c in enumerate(cases):
        sol.set_data(b, *[to_dev(c[k], cuda_dev) for k in ("m_h", "m_l", "w_h", "w_l")])
        if with_truth:
            sol.set_truth(b, to_dev(np.stack([c["truth_c"], c["truth_p"]]), cuda_dev))
    sol._keep = geos
    return sol


@pytest.mark.skipif(not os.path.exists(GOLDEN_EARLY), reason="initial-image oracle pixels for 1024^2 not generated")
def test_full_size_initial_image_float32(cuda_dev):
    # The start decomposes every ray with rho_c = 0 (Eq. 13 without its Compton penalty), where the
    # 2x2 system is ill-conditioned (the Compton and PE columns are nearly parallel, Sec. 1), and its 10
    # float32 PCG iterations on (R^T R + I) x = R^T a_c add the rounding of R / R^T: the full image
    # differs from the FP64 oracle's by 7e-5 relative, the sampled pixels by 2e-4, so the bar is 5e-4
    # (iterations from a common starting image are held below, and from the oracle's start above).
    from paper_1905_00934_gb300 import dect

    ref = json.load(open(GOLDEN_EARLY))
    sl = ref["slices"]
    sol = _mixed_solver(cuda_dev, sl, 0, False)
    sol.reconstruct(0)
    for b, s in enumerate(sl):
        x = sol.get(b, dect.X).cpu().numpy().reshape(2, -1)
        idx = np.array(s["pixels"])
        e_c, e_p = rel_l2(x[0, idx], s["x"][0][0]), rel_l2(x[1, idx], s["x"][0][1])
        assert e_c <= 5e-4 and e_p <= 5e-4, (b, e_c, e_p)


@pytest.fixture(scope="module")
def start_1024():
    """Slice 0 of the 1024 x 1024, 1440-view, 2048-bin workload with float32-rounded measurements, the
    oracle's problem and its initial image rounded to float32 (about a minute on the host cores)."""
    from synth.workloads import BAGGAGE_KAPPA, MIXED_SEED_BASE, baggage_fan_case

    c = baggage_fan_case(slice_index=MIXED_SEED_BASE, n=1024, n_views=1440, n_bins=2048)
    for k in ("m_h", "m_l", "w_h", "w_l"):
        c[k] = _r32(c[k])
    prob = oadmm.Problem(c["geom"], c["spectra"], c["m_h"], c["m_l"], c["w_h"], c["w_l"],
                         oadmm.Params(kappa=BAGGAGE_KAPPA))
    x0 = _r32(np.stack(oadmm.initial_image(prob)))
    return c, prob, x0


@pytest.mark.slow
def test_full_size_iterations_from_the_oracle_initial_image(cuda_dev, start_1024):
    # 1024 x 1024, 1440 views, 2048 bins: the oracle's initial image and 3 ADMM iterations (computed
    # here), the GPU started from that image; the whole images agree to float32 level (measured 2e-6
    # after 3 iterations) until float32 rounding flips a per-ray LM decision, which happens later.
    from paper_1905_00934_gb300 import Geometry, Solver, Spectra, dect
    from synth.workloads import BAGGAGE_KAPPA

    c, prob, x0 = start_1024
    st = oadmm.state_from_image(prob, x0[0], x0[1])
    geo = Geometry(c["geom"])
    sol = Solver([geo], Spectra.from_tables(c["spectra"]), kappa=BAGGAGE_KAPPA)
    sol.set_data(0, *[to_dev(c[k], cuda_dev) for k in ("m_h", "m_l", "w_h", "w_l")], to_dev(x0, cuda_dev))
    sol.reconstruct(0)
    for it in range(1, 4):
        st = oadmm.admm_iteration(prob, st)
        sol.step(1)
        x = sol.get(0, dect.X).cpu().numpy().astype(np.float64)
        e_c, e_p = rel_l2(x[0], st.x[0]), rel_l2(x[1], st.x[1])
        assert e_c <= 5e-5 and e_p <= 5e-5, (it, e_c, e_p)


# After 100 iterations float32 rounding has flipped the accept/reject decision of Eq. 13's LM step
# on near-tied rays (2.9e6 rays per slice); each flip moves that ray by a full step, and these
# perturbations accumulate: with float32 storage the sampled pixels of slice 0 differ from the
# FP64 oracle by 4.3 % (Compton) and 9.0 % (PE) relative L2 while xi (Eq. 14), the quantity the
# workload's error target is set on, tracks the oracle to 0.002 dB at every 10th iteration and
# the rho decisions are identical. The same divergence appears from the oracle's own start and with
# the float64 decomposition (test_full_size_trajectory_from_the_oracle_start: 3.9 % / 7.6 % at 100
# iterations), so it is the float32 state's sensitivity, not the start or the decomposition's
# precision: the trajectory is held on xi and the pixel bound is a regression guard. 16-bit storage
# rounds the stored line integrals (11 / 8 significant bits): measured xi drift over the 4 reference
# slices up to 0.017 dB (float16) and 1.16 dB (bfloat16, slice 3 at iteration 90): bfloat16 storage
# does not hold the workload's 0.5 dB PE-error target on every slice (its bound is a regression
# guard on a format documented as unfit for it), float16 does.
XI_TOL_DB = {0: 0.02, 1: 0.05, 2: 1.5}
PIX_TOL = {0: 0.15, 1: 0.3, 2: 1.0}


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="oracle reference for the 1024^2 workload not generated")
@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "f16", "bf16"])
def test_full_size_subset_against_oracle(cuda_dev, storage):
    from paper_1905_00934_gb300 import dect

    ref = json.load(open(GOLDEN))
    sl = ref["slices"]
    sol = _mixed_solver(cuda_dev, sl, storage, True)
    sol.reconstruct(0)
    worst = 0.0
    for k in range(1, ref["iterations"] // 10 + 1):
        sol.step(10)
        for b, s in enumerate(sl):
            xi = sol.stats(b)["xi_db"]
            d = max(abs(xi[0] - s["xi"][k][0]), abs(xi[1] - s["xi"][k][1]))
            worst = max(worst, d)
            assert d <= XI_TOL_DB[storage], (storage, b, 10 * k, xi, s["xi"][k])
    errs = []
    for b, s in enumerate(sl):
        x = sol.get(b, dect.X).cpu().numpy().reshape(2, -1)
        idx = np.array(s["pixels"])
        errs.append((rel_l2(x[0, idx], s["x_c"]), rel_l2(x[1, idx], s["x_p"])))
    print(f"storage {['f32', 'f16', 'bf16'][storage]}, 1024^2 subset: worst xi difference {worst:.4f} dB, "
          f"sampled-pixel rel-L2 after {ref['iterations']} iterations {errs}")
    assert all(e_c <= PIX_TOL[storage] and e_p <= PIX_TOL[storage] for e_c, e_p in errs)


GOLDEN_FROM_X0 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mixed_1024_from_x0.json")


@pytest.mark.slow
@pytest.mark.skipif(not os.path.exists(GOLDEN_FROM_X0), reason="oracle trajectory from x0 for 1024^2 not generated")
@pytest.mark.parametrize("udm_f64", [0, 1])
def test_full_size_trajectory_from_the_oracle_start(cuda_dev, start_1024, udm_f64):
    """Float32 storage from the oracle's start: sampled pixels after 10, 20, 50 and 100 iterations and
    xi every 10 iterations against the stored FP64 oracle trajectory (tests/golden/mixed_1024_from_x0.json),
    with the float32 decomposition and with the float64 one (udm_f64)."""
    from paper_1905_00934_gb300 import Geometry, Solver, Spectra, dect
    from synth.workloads import BAGGAGE_KAPPA

    c, _, x0 = start_1024
    ref = json.load(open(GOLDEN_FROM_X0))
    idx = np.array(ref["pixels"])
    geo = Geometry(c["geom"])
    sol = Solver([geo], Spectra.from_tables(c["spectra"]), kappa=BAGGAGE_KAPPA, udm_f64=udm_f64)
    sol.set_data(0, *[to_dev(c[k], cuda_dev) for k in ("m_h", "m_l", "w_h", "w_l")], to_dev(x0, cuda_dev))
    sol.set_truth(0, to_dev(np.stack([c["truth_c"], c["truth_p"]]), cuda_dev))
    sol.reconstruct(0)
    errs, xi_worst, done = {}, 0.0, 0
    for k in range(1, 11):
        sol.step(10 * k - done)
        done = 10 * k
        xi = sol.stats(0)["xi_db"]
        xi_worst = max(xi_worst, abs(xi[0] - ref["xi"][k][0]), abs(xi[1] - ref["xi"][k][1]))
        if str(done) in ref["x"]:
            x = sol.get(0, dect.X).cpu().numpy().reshape(2, -1)
            r = ref["x"][str(done)]
            errs[done] = (rel_l2(x[0, idx], r[0]), rel_l2(x[1, idx], r[1]))
    print(f"1024^2 from the oracle start, float32 storage, udm_f64={udm_f64}: sampled-pixel rel-L2 "
          f"(Compton, PE) {errs}; worst xi difference {xi_worst:.4f} dB")
    bounds = TRAJ_PIX_TOL[udm_f64]
    for it, (e_c, e_p) in errs.items():
        assert e_c <= bounds[it] and e_p <= bounds[it], (it, e_c, e_p)
    assert xi_worst <= XI_TOL_DB[0]


# Sampled-pixel bounds per checkpoint (iterations -> relative L2): regression guards at about twice the
# values measured on GB300 from the oracle's own start (float32 decomposition / float64 decomposition):
#   10 its 7.7e-4, 7.1e-4 / 3.4e-4, 3.8e-4;   20 its 7.8e-3, 4.9e-3 / 5.5e-3, 3.7e-3;
#   50 its 2.0e-2, 1.5e-2 / 1.6e-2, 8.8e-3;  100 its 4.0e-2, 8.2e-2 / 3.9e-2, 7.6e-2
# (Compton, PE), xi within 0.0052 / 0.0046 dB of the oracle at every 10th iteration. The float64
# decomposition halves the early difference but leaves the 100-iteration one: what grows is the float32
# rounding of the carried state (R x, a, u^a, the images) that Eq. 13's accept test turns into whole-step
# moves of near-tied rays, and those perturbations compound over the iterations (Sec. 3.3's LM step is a
# discrete decision per ray). The workload's error target is set on xi, which both hold to 0.005 dB.
TRAJ_PIX_TOL = {0: {10: 2e-3, 20: 2e-2, 50: 5e-2, 100: 0.15}, 1: {10: 1e-3, 20: 1.5e-2, 50: 4e-2, 100: 0.15}}
