"""GPU projector R and backprojector R^T against the FP64 oracle (Eq. 2-3's R, Table 1's R^T).

Tolerance: relative L2 <= 1e-5 (float32 accumulation over <= 2N samples per ray / pixel)."""
import math

import numpy as np
import pytest
import torch

from conftest import rel_l2, to_dev
from oracle import projector as oproj
from synth import geometry as G

pytestmark = pytest.mark.gpu

TOL = 1e-5

GEOMS = {
    # several 32x32 backprojector tiles plus ragged tails, non-square, odd sizes, offset detector
    "parallel_ragged": G.Geometry(G.PARALLEL, 53, 37, 0.1, 41, 0.13, math.pi, 77, 0.085, 0.03),
    "parallel_small": G.small_parallel_geometry(),
    "fan_ragged": G.Geometry(G.FAN_FLAT, 45, 61, 0.1, 47, 0.2, 2 * math.pi, 83, 0.13, -0.05, 12.0, 21.0),
    "fan_baggage_128": G.baggage_fan_geometry(128, 180, 256),
    "tiny": G.Geometry(G.PARALLEL, 3, 5, 0.5, 3, 0.3, math.pi, 4, 0.4, 0.0),
    "one_view_one_bin": G.Geometry(G.FAN_FLAT, 9, 9, 0.1, 1, 0.7, 2 * math.pi, 1, 0.2, 0.0, 5.0, 9.0),
    # image much smaller than one tile, source as close as the geometry check allows (4.25 pixels
    # beyond the image's bounding circle plus margin): the tile rectangle must be clipped to the image
    "fan_near_source": G.Geometry(G.FAN_FLAT, 20, 12, 0.1, 64, 0.1, 2 * math.pi, 96, 0.06, 0.0, 1.80, 3.5),
    # three by two tiles with ragged tails, wide detector
    "fan_ragged_tiles": G.Geometry(G.FAN_FLAT, 70, 33, 0.1, 90, 1.1, 2 * math.pi, 140, 0.12, 0.3, 9.0, 15.0),
}


@pytest.fixture(scope="module", params=sorted(GEOMS))
def case(request, cuda_dev):
    from paper_1905_00934_gb300 import Geometry

    g = GEOMS[request.param]
    return g, Geometry(g), cuda_dev


def test_forward_matches_oracle(case):
    g, geo, dev = case
    rng = np.random.default_rng(10)
    x = rng.uniform(0, 1, size=(2, g.ny, g.nx))
    got = geo.project(to_dev(x, dev)).cpu().numpy()
    ref = np.stack([oproj.project(g, x[c]) for c in range(2)])
    assert rel_l2(got, ref) <= TOL
    # one channel: same numbers for channel 0
    got1 = geo.project(to_dev(x[:1], dev)).cpu().numpy()
    assert rel_l2(got1[0], ref[0]) <= TOL


def test_backward_matches_oracle(case):
    g, geo, dev = case
    rng = np.random.default_rng(11)
    y = rng.normal(size=(2, g.n_views, g.n_bins))
    got = geo.backproject(to_dev(y, dev)).cpu().numpy()
    ref = np.stack([oproj.backproject(g, y[c]) for c in range(2)])
    assert rel_l2(got, ref) <= TOL


def test_gpu_pair_is_adjoint(case):
    g, geo, dev = case
    rng = np.random.default_rng(12)
    x = to_dev(rng.normal(size=(2, g.ny, g.nx)), dev)
    y = to_dev(rng.normal(size=(2, g.n_views, g.n_bins)), dev)
    lhs = torch.sum(geo.project(x).double() * y.double()).item()
    rhs = torch.sum(x.double() * geo.backproject(y).double()).item()
    scale = torch.linalg.norm(geo.project(x).double()).item() * torch.linalg.norm(y.double()).item()
    assert abs(lhs - rhs) <= 1e-6 * scale


def test_rays_missing_the_image_are_zero(cuda_dev):
    from paper_1905_00934_gb300 import Geometry

    # detector much wider than the image: outer bins see nothing
    g = G.Geometry(G.PARALLEL, 8, 8, 0.1, 6, 0.0, math.pi, 40, 0.1, 0.0)
    x = np.ones((1, 8, 8))
    got = Geometry(g).project(to_dev(x, cuda_dev)).cpu().numpy()[0]
    ref = oproj.project(g, x[0])
    assert np.all(ref[:, :5] == 0) and np.all(got[:, :5] == 0)
    assert rel_l2(got, ref) <= TOL


def test_deterministic(cuda_dev):
    from paper_1905_00934_gb300 import Geometry

    g = GEOMS["fan_ragged"]
    geo = Geometry(g)
    rng = np.random.default_rng(13)
    y = to_dev(rng.normal(size=(2, g.n_views, g.n_bins)), cuda_dev)
    a = geo.backproject(y).cpu().numpy()
    b = geo.backproject(y).cpu().numpy()
    assert np.array_equal(a, b)


def test_full_size_baggage_fan(cuda_dev):
    # the 512 x 512, 720 x 1024 fan-beam workload at full size, in the launch configuration the solver uses
    from paper_1905_00934_gb300 import Geometry
    from synth.workloads import baggage_fan_case

    c = baggage_fan_case()
    g = c["geom"]
    geo = Geometry(g)
    x = np.stack([c["truth_c"], c["truth_p"]])
    got = geo.project(to_dev(x, cuda_dev)).cpu().numpy()
    ref = np.stack([oproj.project(g, x[ch]) for ch in range(2)])
    assert rel_l2(got[0], ref[0]) <= TOL and rel_l2(got[1], ref[1]) <= TOL
    rng = np.random.default_rng(14)
    y = rng.normal(size=(2, g.n_views, g.n_bins))
    gotb = geo.backproject(to_dev(y, cuda_dev)).cpu().numpy()
    refb = np.stack([oproj.backproject(g, y[ch]) for ch in range(2)])
    assert rel_l2(gotb, refb) <= TOL


@pytest.mark.slow
def test_largest_workload_geometry(cuda_dev):
    # the largest workload's geometry (1024 x 1024 fan, 1440 views x 2048 bins): R and R^T through the
    # single-slice entry points, and R through the batched solver, whose two slices of one geometry are
    # projected by one CTA (the initial state of a solver given start images holds R x0)
    from paper_1905_00934_gb300 import Geometry, Solver, Spectra, dect
    from synth.spectra import SpectralTables

    g = G.baggage_fan_geometry(1024, 1440, 2048)
    geo = Geometry(g)
    rng = np.random.default_rng(31)
    x = rng.uniform(0.0, 1.0, size=(2, g.ny, g.nx)).astype(np.float32).astype(np.float64)
    ref = np.stack([oproj.project(g, x[ch]) for ch in range(2)])
    got = geo.project(to_dev(x, cuda_dev)).cpu().numpy()
    assert rel_l2(got[0], ref[0]) <= TOL and rel_l2(got[1], ref[1]) <= TOL
    y = rng.normal(size=(2, g.n_views, g.n_bins)).astype(np.float32).astype(np.float64)
    refb = np.stack([oproj.backproject(g, y[ch]) for ch in range(2)])
    gotb = geo.backproject(to_dev(y, cuda_dev)).cpu().numpy()
    assert rel_l2(gotb[0], refb[0]) <= TOL and rel_l2(gotb[1], refb[1]) <= TOL

    sol = Solver([geo, geo], Spectra.from_tables(SpectralTables(e_ref_kev=100.0)), proj_views=2)
    zero = torch.zeros((g.n_views, g.n_bins), dtype=torch.float32, device=cuda_dev)
    one = torch.ones_like(zero)
    for b, img in enumerate((x, x[::-1].copy())):  # the second slice: the channels swapped
        sol.set_data(b, zero, zero, one, one, to_dev(img, cuda_dev))
    sol.reconstruct(0)
    torch.cuda.synchronize()
    for b, r in enumerate((ref, ref[::-1])):
        rx = sol.get(b, dect.RX).cpu().numpy()
        assert rel_l2(rx[0], r[0]) <= TOL and rel_l2(rx[1], r[1]) <= TOL, b
