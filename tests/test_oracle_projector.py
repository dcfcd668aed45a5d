"""Pins for the oracle's projector R and backprojector R^T (Eq. 2-3's R, Table 1's R^T)."""
import math

import numpy as np
import pytest

from oracle import projector
from synth import geometry as G
from synth import phantom as P


def _disk_phantom(r, c=0.3, p=0.0, cx=0.0, cy=0.0):
    return P.Phantom(np.array([P.ELLIPSE]), np.array([cx]), np.array([cy]), np.array([r]), np.array([r]),
                     np.array([0.0]), np.array([c]), np.array([p]))


def _mixed_phantom():
    return P.Phantom(np.array([P.ELLIPSE, P.ELLIPSE, P.RECTANGLE]), np.array([0.0, 0.8, -0.9]),
                     np.array([0.0, -0.5, 0.7]), np.array([2.6, 0.9, 0.6]), np.array([2.2, 0.5, 0.9]),
                     np.array([0.3, 1.1, 0.4]), np.array([0.2, 0.15, 0.1]), np.array([0.0, 0.0, 0.0]))


def test_parallel_zero_angle_is_column_sums():
    # theta = 0: vertical rays through the column centres; weight = pixel size per row
    g = G.parallel_geometry(16, 4, 16, 0.1, 0.1, span_rad=2 * math.pi)
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(16, 16))
    s = projector.project(g, x)
    assert np.allclose(s[0], 0.1 * x.sum(axis=0), rtol=1e-13)       # theta = 0
    assert np.allclose(s[1], 0.1 * x.sum(axis=1), rtol=1e-13)       # theta = pi/2: row sums
    assert np.allclose(s[2], 0.1 * x.sum(axis=0)[::-1], rtol=1e-13)  # theta = pi (u flips)


def test_constant_image_gives_chord_length_for_edge_to_edge_rays():
    # a ray that enters and leaves through the two opposite sides it is sampled along
    # collects exactly (number of columns) * pix / |d_major| = its chord through the square
    g = G.parallel_geometry(32, 37, 48, 0.1, 0.07)
    x = np.ones((32, 32))
    s = projector.project(g, x)
    px, py, dx, dy = g.rays()
    half = 0.5 * (32 - 1) * 0.1
    checked = 0
    for v in range(g.n_views):
        for k in range(g.n_bins):
            if abs(dx[v, k]) >= abs(dy[v, k]):
                ya = py[v, k] + (-half - px[v, k]) * dy[v, k] / dx[v, k]
                yb = py[v, k] + (half - px[v, k]) * dy[v, k] / dx[v, k]
                if max(abs(ya), abs(yb)) <= half:
                    assert s[v, k] == pytest.approx(32 * 0.1 / abs(dx[v, k]), rel=1e-12)
                    checked += 1
            else:
                xa = px[v, k] + (-half - py[v, k]) * dx[v, k] / dy[v, k]
                xb = px[v, k] + (half - py[v, k]) * dx[v, k] / dy[v, k]
                if max(abs(xa), abs(xb)) <= half:
                    assert s[v, k] == pytest.approx(32 * 0.1 / abs(dy[v, k]), rel=1e-12)
                    checked += 1
    assert checked > 200


@pytest.mark.parametrize("kind", ["parallel", "fan"])
def test_converges_to_analytic_radon_transform(kind):
    # R applied to the pixelised phantom approaches the exact line integrals as pixels shrink
    errs = []
    ph = _mixed_phantom()
    for n in (32, 64, 128, 256):
        pix = 6.4 / n
        if kind == "parallel":
            g = G.parallel_geometry(n, 45, 96, pix, 0.1)
        else:
            g = G.Geometry(G.FAN_FLAT, n, n, pix, 45, 0.1, 2 * math.pi, 96, 0.12, 0.0, 12.0, 20.0)
        xc, _ = P.truth_image(ph, g, supersample=8)
        exact, _ = P.line_integrals(ph, g)
        errs.append(np.linalg.norm(projector.project(g, xc) - exact) / np.linalg.norm(exact))
    errs = np.array(errs)
    assert errs[-1] < 5e-3
    assert np.all(errs[1:] < errs[:-1])
    # observed order at least 1 under refinement (piecewise-constant objects)
    assert errs[0] / errs[-1] > 6.0


def test_fan_central_ray_through_disk_is_its_diameter():
    g = G.Geometry(G.FAN_FLAT, 128, 128, 0.05, 8, 0.0, 2 * math.pi, 65, 0.1, 0.0, 10.0, 18.0)
    ph = _disk_phantom(2.0, c=1.0)
    exact, _ = P.line_integrals(ph, g)
    assert np.allclose(exact[:, 32], 4.0, rtol=1e-12)  # bin 32 of 65 is the central ray
    xc, _ = P.truth_image(ph, g, supersample=8)
    s = projector.project(g, xc)
    assert np.allclose(s[:, 32], 4.0, rtol=1e-2)  # pixelisation of the disk edge


@pytest.mark.parametrize("kind", ["parallel", "fan"])
def test_adjoint_identity(kind):
    rng = np.random.default_rng(1)
    if kind == "parallel":
        g = G.parallel_geometry(40, 33, 57, 0.1, 0.09, angle0_rad=0.05)
    else:
        g = G.Geometry(G.FAN_FLAT, 40, 36, 0.1, 31, 0.2, 2 * math.pi, 61, 0.13, 0.02, 9.0, 15.0)
    x = rng.normal(size=(g.ny, g.nx))
    y = rng.normal(size=(g.n_views, g.n_bins))
    lhs = np.vdot(projector.project(g, x), y)
    rhs = np.vdot(x, projector.backproject(g, y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs) + 1e-12


@pytest.mark.parametrize("kind", ["parallel", "fan"])
def test_explicit_matrix_transpose_on_8x8(kind):
    if kind == "parallel":
        g = G.parallel_geometry(8, 7, 12, 0.1, 0.1, angle0_rad=0.1)
    else:
        g = G.Geometry(G.FAN_FLAT, 8, 8, 0.1, 9, 0.0, 2 * math.pi, 13, 0.11, 0.0, 3.0, 5.0)
    Rm = projector.matrix(g)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(8, 8))
    y = rng.normal(size=(g.n_views, g.n_bins))
    assert np.allclose(Rm @ x.ravel(), projector.project(g, x).ravel(), rtol=1e-13, atol=1e-14)
    assert np.allclose(Rm.T @ y.ravel(), projector.backproject(g, y).ravel(), rtol=1e-13, atol=1e-14)
    # every weight is non-negative and at most pix / |d_major| <= pix * sqrt(2)
    assert Rm.min() >= 0.0 and Rm.max() <= 0.1 * math.sqrt(2) + 1e-15


def test_single_ray_matches_full_projection():
    g = G.baggage_fan_geometry(64, 36, 80)
    rng = np.random.default_rng(3)
    x = rng.uniform(size=(64, 64))
    s = projector.project(g, x)
    for v, k in [(0, 0), (5, 40), (35, 79), (17, 33)]:
        assert projector.project_ray(g, x, v, k) == s[v, k]
