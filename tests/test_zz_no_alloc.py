"""tet_render_noalloc, the entry point for callers that may not let a library
allocate device memory: through the C ABI it gives the same image as
tet_render and as the CPU oracle (within the render tests' per-pixel
tolerance) on two calls in a row, the second reusing the static scratch array
the first one left behind; a call after the first changes the device's free
memory by nothing; and it refuses a frame larger than that array."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from paper_2506_11510_gb300 import _native as N
from paper_2506_11510_gb300 import api, workloads as W
from tests.conftest import scene_volume

pytestmark = pytest.mark.gpu


def test_noalloc_render_matches_tet_render_twice():
    s = W.scene("tiny")
    vol = torch.from_numpy(scene_volume("tiny")).cuda()
    grid = api.build_scene_grid(s, vol)
    ref, ref2 = api.tet_render(grid, s.camera, s.medium, s.spp, s.render_seed)
    orc, orc2, _ = O.Grid.for_scene(s, scene_volume("tiny")).render(s.camera, s.medium, s.spp, s.render_seed)
    cam, med = api.camera_struct(s.camera), api.medium_struct(s.medium)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def close(a, b):
        return np.mean(np.abs(a - b) <= 1e-4 * np.maximum(np.abs(b), 1e-5) + 1e-6)

    outs = [(torch.zeros_like(ref), torch.zeros_like(ref)) for _ in range(2)]
    torch.cuda.synchronize()
    for k, (out, out2) in enumerate(outs):
        free0 = torch.cuda.mem_get_info()[0]
        st = N.lib().tet_render_noalloc(grid.handle, C.byref(cam), C.byref(med), s.spp, C.c_uint64(s.render_seed),
                                        0, C.c_void_p(out.data_ptr()), C.c_void_p(out2.data_ptr()), stream)
        assert st == N.TG_OK
        torch.cuda.synchronize()
        if k > 0:
            # the entry point's defining property: no device memory is taken by the call
            assert torch.cuda.mem_get_info()[0] == free0
        g, g2 = out.cpu().numpy().astype(np.float64), out2.cpu().numpy().astype(np.float64)
        assert close(g, ref.cpu().numpy().astype(np.float64)) >= 0.999
        assert close(g2, ref2.cpu().numpy().astype(np.float64)) >= 0.999
        # and the image is the oracle's (fp64, the same Philox streams)
        assert close(g, orc) >= 0.999
        assert close(g2, orc2) >= 0.999


def test_noalloc_rejects_frames_beyond_its_scratch():
    s = W.scene("tiny")
    vol = torch.from_numpy(scene_volume("tiny")).cuda()
    grid = api.build_scene_grid(s, vol)
    big = W.Camera(s.camera.pos, s.camera.target, s.camera.up, s.camera.fov_y_deg, 1024, 1024)
    out = torch.zeros((1024, 1024), device="cuda")
    st = N.lib().tet_render_noalloc(grid.handle, C.byref(api.camera_struct(big)), C.byref(api.medium_struct(s.medium)),
                                    1, C.c_uint64(1), 0, C.c_void_p(out.data_ptr()), None, None)
    assert st == N.TG_EINVAL
