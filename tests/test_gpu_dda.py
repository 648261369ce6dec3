"""The regular-grid comparator on the GPU (3D DDA, same estimator) against the
oracle's voxel walker: per-path estimates and images."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2506_11510_gb300 import workloads as W
from tests.conftest import scene_volume
from tests.test_gpu_render import FRAC, REL, all_paths

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["tiny", "adaptive_small"])
def test_dda_paths_match_oracle(name):
    import paper_2506_11510_gb300 as tv
    s = W.scene(name)
    vol = scene_volume(name)
    px, py, sm = all_paths(s.camera, s.spp)
    got = tv.grid_trace_paths(torch.from_numpy(vol).cuda(), s.box_min, s.voxel_size, s.camera, s.medium,
                              s.render_seed, px, py, sm)
    want = O.dda_render_paths(vol, s.box_min, s.voxel_size, s.camera, s.medium, s.render_seed, px, py, sm)
    L = got["L"].cpu().numpy().astype(np.float64)
    close = np.abs(L - want["L"]) <= REL * np.maximum(np.abs(want["L"]), 1e-6)
    assert close.mean() >= FRAC, close.mean()
    assert np.mean(got["collisions"].cpu().numpy() == want["collisions"]) >= FRAC


def test_dda_image_matches_oracle():
    import paper_2506_11510_gb300 as tv
    s = W.scene("tiny")
    vol = scene_volume("tiny")
    img, _ = tv.grid_render(torch.from_numpy(vol).cuda(), s.box_min, s.voxel_size, s.camera, s.medium, s.spp,
                            s.render_seed)
    ref, _, _ = O.dda_render(vol, s.box_min, s.voxel_size, s.camera, s.medium, s.spp, s.render_seed)
    g = img.cpu().numpy().astype(np.float64)
    close = np.abs(g - ref) <= 1e-4 * np.maximum(np.abs(ref), 1e-5) + 1e-6
    assert close.mean() >= 0.999
