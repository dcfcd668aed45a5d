"""The projector entry point that allocates nothing (dect_project_noalloc).

It is meant for callers that cannot allocate device memory, such as code running
while a CUDA stream is being captured or code whose device memory is owned by its own
pool. Its scratch is a fixed array inside the library, shared by all calls. This test
calls it through the C ABI twice in a row, with different images, and checks both
results against dect_project (the allocating entry point) with the projector
tolerance used elsewhere (relative L2 <= 1e-5), so a stale texture from the first
call would show up in the second. It also checks that an image too large for the
fixed scratch is refused with a message. The file name makes pytest collect it last.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from conftest import rel_l2, to_dev
from synth import geometry as G

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.mark.parametrize("g", [G.Geometry(G.PARALLEL, 128, 128, 0.1, 90, 0.0, math.pi, 181, 0.1),
                               G.Geometry(G.FAN_FLAT, 96, 80, 0.1, 60, 0.3, 2 * math.pi, 150, 0.12, 0.0,
                                          14.0, 24.0)],
                         ids=["parallel_128", "fan_96x80"])
def test_noalloc_projection_matches_dect_project_on_two_calls(cuda_dev, g):
    from paper_1905_00934_gb300 import Geometry, dect

    geo = Geometry(g)
    rng = np.random.default_rng(7)
    x1 = to_dev(rng.uniform(0, 1, (2, g.ny, g.nx)), cuda_dev)
    x2 = to_dev(rng.uniform(0, 3, (2, g.ny, g.nx)), cuda_dev)
    out1 = torch.empty((2, g.n_views, g.n_bins), dtype=torch.float32, device=cuda_dev)
    out2 = torch.empty_like(out1)
    dect.project_noalloc(geo.handle, x1, out1)
    dect.project_noalloc(geo.handle, x2, out2)
    ref1 = geo.project(x1)
    ref2 = geo.project(x2)
    torch.cuda.synchronize()
    assert rel_l2(out1.cpu().numpy(), ref1.cpu().numpy()) <= TOL
    assert rel_l2(out2.cpu().numpy(), ref2.cpu().numpy()) <= TOL
    # one channel uses the same scratch layout
    o1 = torch.empty((1, g.n_views, g.n_bins), dtype=torch.float32, device=cuda_dev)
    dect.project_noalloc(geo.handle, x1[:1].contiguous(), o1)
    torch.cuda.synchronize()
    assert rel_l2(o1.cpu().numpy()[0], ref1.cpu().numpy()[0]) <= TOL


def test_noalloc_rejects_images_beyond_the_fixed_scratch(cuda_dev):
    from paper_1905_00934_gb300 import Geometry, dect

    g = G.Geometry(G.PARALLEL, 400, 400, 0.1, 8, 0.0, math.pi, 16, 0.1)
    geo = Geometry(g)
    x = torch.zeros((1, 400, 400), dtype=torch.float32, device=cuda_dev)
    out = torch.zeros((1, 8, 16), dtype=torch.float32, device=cuda_dev)
    status = dect.lib().dect_project_noalloc(geo.handle, 1, ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()), None)
    assert status == dect.EINVAL
    assert b"scratch" in dect.lib().dect_last_error()
