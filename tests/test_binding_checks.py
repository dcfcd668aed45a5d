"""The binding refuses tensors whose dtype, shape or device do not match what a C entry point will
read or write through its plain pointers (checked before any library call, so on any host)."""
import types

import pytest
import torch

from paper_1905_00934_gb300 import dect

# a geometry's shape (nx 8, ny 6, 5 views, 7 bins); no handle is needed, the checks come first
G = types.SimpleNamespace(handle=None, nx=8, ny=6, n_views=5, n_bins=7)
z = torch.zeros


def test_project_and_backproject_refuse_mismatches():
    with pytest.raises(TypeError):  # a float64 image into a float32 sinogram
        dect.project(G, z(2, 6, 8, dtype=torch.float64), z(2, 5, 7))
    with pytest.raises(TypeError):
        dect.backproject(G, z(2, 5, 7, dtype=torch.float64), z(2, 6, 8))
    with pytest.raises(TypeError):
        dect.project(G, z(2, 6, 8, dtype=torch.float16), z(2, 5, 7, dtype=torch.float16))
    with pytest.raises(ValueError):  # transposed image
        dect.project(G, z(2, 8, 6), z(2, 5, 7))
    with pytest.raises(ValueError):  # sinogram of another geometry
        dect.backproject(G, z(2, 7, 5), z(2, 6, 8))
    with pytest.raises(ValueError):  # three channels
        dect.project(G, z(3, 6, 8), z(3, 5, 7))
    with pytest.raises(ValueError):  # channel counts differ
        dect.project(G, z(2, 6, 8), z(1, 5, 7))
    with pytest.raises(ValueError):  # not contiguous
        dect.project(G, z(2, 6, 16)[:, :, ::2], z(2, 5, 7))
    with pytest.raises(ValueError):  # host memory
        dect.project(G, z(2, 6, 8), z(2, 5, 7))
    with pytest.raises(TypeError):
        dect.project(G, [0.0], z(2, 5, 7))


def test_fbp_takes_float32_only():
    with pytest.raises(TypeError):
        dect.fbp(G, z(1, 5, 7, dtype=torch.float64), z(1, 6, 8, dtype=torch.float64))
    with pytest.raises(ValueError):
        dect.fbp(G, z(1, 5, 7), z(1, 8, 6))


def test_solver_inputs_are_sized():
    m = z(35)
    with pytest.raises(ValueError):  # one measurement array short
        dect.admm_set_data(None, 0, m, m, m, z(34), n_rays=35, n_pix=48)
    with pytest.raises(TypeError):
        dect.admm_set_data(None, 0, m, m, m, z(35, dtype=torch.float64), n_rays=35, n_pix=48)
    with pytest.raises(ValueError):  # a start image of one basis only
        dect.admm_set_data(None, 0, m, m, m, m, z(48), n_rays=35, n_pix=48)
    with pytest.raises(ValueError):
        dect.admm_set_truth(None, 0, z(2, 6, 7), n_pix=48)


def test_per_ray_calls_are_sized():
    a = z(9)
    with pytest.raises(ValueError):
        dect.decompose_rays(None, a, a, a, a, a, a, 1e-3, 1e-3, 1, a, z(8), a)
    with pytest.raises(TypeError):
        dect.decompose_rays(None, a, a, a, a, a, a, 1e-3, 1e-3, 1, a, a, a, z(9))  # status must be uint8
    with pytest.raises(TypeError):
        dect.forward_model(None, a, z(9, dtype=torch.float64))
    with pytest.raises(ValueError):
        dect.forward_model(None, a, a, jac=z(9, 3))
    with pytest.raises(ValueError):
        dect.forward_model_vjp(None, a, a, a, a, a, z(10))


def test_cdm_fbp_is_sized():
    m = z(35)
    with pytest.raises(ValueError):  # measurements of another geometry
        dect.cdm_fbp(G, None, z(34), z(34), z(34), z(34), 5, z(2, 6, 8))
    with pytest.raises(ValueError):  # one image where the method writes two
        dect.cdm_fbp(G, None, m, m, m, m, 5, z(1, 6, 8))
    with pytest.raises(ValueError):
        dect.cdm_fbp(G, None, m, m, m, m, 5, z(2, 6, 8), work=z(35))


def test_solver_data_sizes_follow_the_first_array():
    with pytest.raises(ValueError):
        dect.admm_set_data(None, 0, z(35), z(35), z(36), z(35))


def test_unknown_solver_parameters_are_refused():
    with pytest.raises(TypeError):
        dect.params_default(bp_view_group=4)  # a misspelt field would otherwise be dropped
    assert dect.params_default(bp_view_groups=4).bp_view_groups == 4
