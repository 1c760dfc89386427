"""vpgs_render_fwd_noalloc, the render for callers that cannot allocate device memory.

Such callers (a plugin given only a stream and tensors, a process whose memory
pool owns the GPU) get the same render through a scratch array compiled into
the library.  Its output must match the workspace entry point's, call after
call.  This file is collected last so a failure here cannot hide the other
tests.
"""
import ctypes

import pytest
import torch

from paper_2505_18992_gb300 import scenes
from paper_2505_18992_gb300 import vpgs as C
from paper_2505_18992_gb300.build import build
from paper_2505_18992_gb300.render import Intrinsics, Renderer, current_stream_handle
from tests.helpers import FWD_ATOL, intrinsics, scene_tensors

pytestmark = pytest.mark.gpu


def test_noalloc_render_matches_the_workspace_render_twice():
    build()
    sc = scenes.tiny_planes()  # 10,000 Gaussians at 320x240 fit the 32 MiB array
    r = Renderer(intrinsics(sc))
    g, T = scene_tensors(sc)
    ref = r.forward(*g, T)
    torch.cuda.synchronize()
    gs = r._gauss(*g)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        out = r.alloc_images()
        code = C.vpgs_render_fwd_noalloc(ctypes.byref(gs), ctypes.byref(r.cam), T.data_ptr(), 1,
                                         ctypes.byref(r.opts), ctypes.byref(r._images(out)),
                                         status.data_ptr(), current_stream_handle())
        assert code == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        for k in ("rgb", "depth", "alpha", "t_final"):
            assert float((out[k] - ref[k]).abs().max()) <= FWD_ATOL, k
        for k in ("n_contrib", "n_iter"):
            assert torch.equal(out[k], ref[k]), k
        status.fill_(-1)


def test_noalloc_render_rejects_a_request_beyond_its_scratch():
    build()
    n = 2_000_000  # its smallest workspace is far above 32 MiB
    z = torch.zeros((n, 4), device="cuda")
    gs = C.vpgs_gaussians(z.data_ptr(), z.data_ptr(), z.data_ptr(), z.data_ptr(), z.data_ptr(), n, None)
    cam = C.vpgs_camera(320, 240, 300.0, 300.0, 160.0, 120.0)
    opts = C.default_opts()
    T = torch.eye(4, dtype=torch.float64, device="cuda")[None].contiguous()
    out = Renderer(Intrinsics(320, 240, 300.0, 300.0, 160.0, 120.0)).alloc_images()
    code = C.vpgs_render_fwd_noalloc(ctypes.byref(gs), ctypes.byref(cam), T.data_ptr(), 1,
                                     ctypes.byref(opts), ctypes.byref(Renderer._images(out)), None,
                                     current_stream_handle())
    assert code == 6


def test_noalloc_render_reports_tile_instances_beyond_its_scratch():
    """The Gaussians' own arrays fit the scratch, but their tile instances do
    not: the call is accepted and the device status reads VPGS_ERR_CAPACITY."""
    build()
    sc = scenes.random_gaussians(20_000, 320, 240, 300.0, seed=4, depth=(1.5, 2.0), spread=0.2,
                                 scale_range=(0.5, 0.8))  # each covers most of the image's 300 tiles
    r = Renderer(intrinsics(sc))
    g, T = scene_tensors(sc)
    gs = r._gauss(*g)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    out = r.alloc_images()
    code = C.vpgs_render_fwd_noalloc(ctypes.byref(gs), ctypes.byref(r.cam), T.data_ptr(), 1,
                                     ctypes.byref(r.opts), ctypes.byref(r._images(out)),
                                     status.data_ptr(), current_stream_handle())
    assert code == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 2
