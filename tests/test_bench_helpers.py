"""The bench's algorithmic-work counter: the number of non-zero weights of R (Eq. 2-3's projection
matrix) that the roofline is computed from, against the oracle's explicit matrix on small geometries."""
import math

import numpy as np
import pytest

import bench
from oracle import projector
from synth import geometry as G


@pytest.mark.parametrize("g", [
    G.Geometry(G.FAN_FLAT, 13, 11, 0.1, 17, 0.2, 2 * math.pi, 23, 0.13, 0.01, 5.0, 9.0),
    G.Geometry(G.FAN_FLAT, 20, 20, 0.1, 30, 0.05, 2 * math.pi, 31, 0.11, -0.02, 7.0, 12.0),
    G.Geometry(G.PARALLEL, 16, 9, 0.1, 21, 0.07, math.pi, 25, 0.083, 0.01),
], ids=["fan_small", "fan_square", "parallel_offset"])
def test_weight_count_equals_the_explicit_matrix(g):
    # off-grid geometries: no sample lands exactly on a pixel centre, so every counted weight is non-zero
    assert bench.joseph_weight_count(g) == np.count_nonzero(projector.matrix(g))


def test_weight_count_grows_with_the_workload():
    small = G.fan_geometry(64, 90, 128)
    large = G.fan_geometry(128, 180, 256)
    ratio = bench.joseph_weight_count(large) / bench.joseph_weight_count(small)
    assert 7.0 < ratio < 9.0  # views x bins x samples per ray: ~2 x 2 x 2


def test_stored_oracle_values_load():
    # the quality gate and the CDM-FBP comparison read these files written by tests/golden scripts
    import bench

    gold = bench._golden()
    assert gold is not None and len(gold["xi_p"]) == bench.ITERS + 1
    cdm = bench._golden(bench.GOLDEN_CDM_FBP)
    assert cdm is not None and cdm["decomposition_iterations"] == bench.CDM_ITERS
    assert set(cdm) >= {"xi_c", "xi_p"}
