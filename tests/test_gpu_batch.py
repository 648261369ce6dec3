"""Batched heterogeneous rendering (one persistent launch over many grids,
cameras, media and images, replayed as a CUDA graph): every job's image equals
what tet_render adds for that job alone, with and without the autotuner, and
the per-job completion times are reported."""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2506_11510_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _jobs(n, seed, max_dim=96):
    import paper_2506_11510_gb300 as tv
    out = []
    for s in W.batch_scenes(n, seed=seed, max_dim=max_dim):
        s = W.with_camera(s, width=min(s.camera.width, 160), height=min(s.camera.height, 144))
        s = dataclasses.replace(s, spp=min(s.spp, 8))
        vol = W.make_volume(s, device="cuda")
        grid = tv.build_scene_grid(s, vol)
        out.append((s, grid))
    return out


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_images_equal_single_renders(autotune):
    import paper_2506_11510_gb300 as tv
    jobs = _jobs(7, 300 + int(autotune))
    imgs = [(torch.zeros((s.camera.height, s.camera.width), device="cuda"),
             torch.zeros((s.camera.height, s.camera.width), device="cuda")) for s, _ in jobs]
    b = tv.Batch([(g, s.camera, s.medium, s.spp, s.render_seed, a, a2) for (s, g), (a, a2) in zip(jobs, imgs)],
                 autotune=autotune)
    b.render()
    b.render()                                     # a second frame: the graph replays and adds again
    torch.cuda.synchronize()
    for (s, g), (a, a2) in zip(jobs, imgs):
        r, r2 = tv.tet_render(g, s.camera, s.medium, s.spp, s.render_seed)
        want, want2 = 2 * r.double(), 2 * r2.double()
        got, got2 = a.double(), a2.double()
        # the same paths; only the order of the per-pixel float atomics differs
        assert torch.allclose(got, want, rtol=1e-5, atol=1e-6)
        assert torch.allclose(got2, want2, rtol=1e-5, atol=1e-6)
        assert float(want.sum()) > 0
    knobs, ms = b.info()
    assert knobs["regen_min"] in (4, 8, 16) and knobs["ev_min"] in (8, 12, 16) and knobs["order"] in (0, 1)
    assert len(ms) == 7 and all(0 < t < 60000 for t in ms)


def test_batch_rejects_mixed_density_formats():
    import paper_2506_11510_gb300 as tv
    from paper_2506_11510_gb300 import TetvolError
    (s, g), = _jobs(1, 400)
    s2 = W.scene("production_small")
    g2 = tv.build_scene_grid(s2, W.make_volume(s2, device="cuda"))
    a = torch.zeros((s.camera.height, s.camera.width), device="cuda")
    a2 = torch.zeros((s2.camera.height, s2.camera.width), device="cuda")
    with pytest.raises(TetvolError):
        tv.Batch([(g, s.camera, s.medium, 2, 1, a, None), (g2, s2.camera, s2.medium, 2, 1, a2, None)])
