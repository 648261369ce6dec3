"""Batched heterogeneous rendering (one persistent launch over many grids,
cameras, media and images, replayed as a CUDA graph): every job's image is the
fp64 oracle's image of that job (grid, camera, medium, seed and sample range),
and equals what tet_render adds for that job alone, with and without the
autotuner; the per-job completion times are reported."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from paper_2506_11510_gb300 import workloads as W
from tests.test_gpu_render import FRAC, REL

pytestmark = pytest.mark.gpu


def _jobs(n, seed, max_dim=96, g_mix=False, volumes=None):
    import paper_2506_11510_gb300 as tv
    out = []
    for k, s in enumerate(W.batch_scenes(n, seed=seed, max_dim=max_dim)):
        s = W.with_camera(s, width=min(s.camera.width, 160), height=min(s.camera.height, 144))
        s = dataclasses.replace(s, spp=min(s.spp, 8))
        if g_mix and k < 2:
            s = W.with_medium(s, g=(-0.25, 0.7)[k])       # both signs of g in every batch
        vol = W.make_volume(s, device="cuda")
        grid = tv.build_scene_grid(s, vol)
        if volumes is not None:
            volumes.append(vol.cpu().numpy())
        out.append((s, grid))
    return out


def test_batch_images_match_the_oracle():
    """Each job of one batched launch against the oracle's render of that job:
    per-pixel sums within 1e-4 relative (floor 1e-5, plus 1e-6) for all but the
    pixels that hold one of the <= 0.1% of paths allowed to differ (at most
    spp * 0.1% of the pixels), and each image's mean inside 3 sd / sqrt(n) of
    the oracle's.  The jobs differ in grid size, view, spp, albedo and g (both
    signs), so a wrong per-job parameter or job selection shows in some image."""
    import paper_2506_11510_gb300 as tv
    vols = []
    jobs = _jobs(6, 310, g_mix=True, volumes=vols)
    assert min(s.medium.g for s, _ in jobs) < 0 < max(s.medium.g for s, _ in jobs)
    imgs = [(torch.zeros((s.camera.height, s.camera.width), device="cuda"),
             torch.zeros((s.camera.height, s.camera.width), device="cuda")) for s, _ in jobs]
    b = tv.Batch([(g, s.camera, s.medium, s.spp, s.render_seed, a, a2) for (s, g), (a, a2) in zip(jobs, imgs)])
    b.render()
    torch.cuda.synchronize()
    for (s, _), (a, a2), vnp in zip(jobs, imgs, vols):
        osum, osq, _ = O.Grid.for_scene(s, vnp).render(s.camera, s.medium, s.spp, s.render_seed)
        got, got2 = a.cpu().numpy().astype(np.float64), a2.cpu().numpy().astype(np.float64)
        close = np.abs(got - osum) <= REL * np.maximum(np.abs(osum), 1e-5) + 1e-6
        assert close.mean() >= 1 - s.spp * (1 - FRAC), (s.name, close.mean())
        close2 = np.abs(got2 - osq) <= REL * np.maximum(np.abs(osq), 1e-5) + 1e-6
        assert close2.mean() >= 1 - s.spp * (1 - FRAC), (s.name, close2.mean())
        # image mean: per-pixel differences average out (3 sd / sqrt(n))
        d = (got - osum).ravel()
        if d.std() > 0:
            assert abs(d.mean()) <= 3 * d.std() / np.sqrt(d.size) + 1e-7
    b.free()


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
