"""Extra channels and the voxel medium on the GPU against the oracle: channel
means and voxel majorants bit for bit, per-path estimates of the extended
estimator (emission, per-cell albedo and g, delta tracking against the cell
majorants with ratio-tracked shadows) within 1e-4 for >= 99.9% of paths, the
frame against its own paths, the furnace, and the tet-majorant delta tracker
against the GPU regular-grid comparator on the same voxel medium."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2506_11510_gb300 import workloads as W
from tests.conftest import scene_volume
from tests.test_gpu_render import all_paths

pytestmark = pytest.mark.gpu

EMISSION, ALBEDO, GCHAN, VOXEL = 1, 2, 4, 8
REL, FRAC = 1e-4, 0.999


def _pair(name):
    import paper_2506_11510_gb300 as tv
    s = W.scene(name)
    vol = scene_volume(name)
    t, a, g = W.make_channels(s)
    grid = tv.build_scene_grid(s, torch.from_numpy(vol).cuda())
    grid.channels(torch.from_numpy(vol).cuda(), t.cuda(), a.cuda(), g.cuda())
    ref = O.Grid.for_scene(s, vol)
    ref.channels(vol, t.numpy(), a.numpy(), g.numpy())
    return s, vol, grid, ref


@pytest.fixture(scope="module")
def small():
    return _pair("adaptive_small")


@pytest.mark.parametrize("name", ["tiny", "adaptive_small", "production_small"])
def test_channels_and_majorants_bit_exact(name):
    s, vol, grid, ref = _pair(name)
    chan, vmaj = grid.export_channels()
    oc, ov = ref.export_channels()
    assert np.array_equal(chan[:, :3].cpu().numpy(), oc)
    assert np.all(chan[:, 3].cpu().numpy() == 0)
    assert np.array_equal(vmaj.cpu().numpy(), ov)


@pytest.mark.parametrize("flags", [EMISSION | ALBEDO | GCHAN, VOXEL, VOXEL | EMISSION | ALBEDO | GCHAN])
def test_extended_paths_match_oracle(small, flags):
    import paper_2506_11510_gb300 as tv
    s, vol, grid, ref = small
    px, py, sm = all_paths(s.camera, 1)
    med = W.with_medium(s, sigma_scale=48.0).medium
    dv = torch.from_numpy(vol).cuda()
    got = tv.tet_trace_ext_paths(grid, s.camera, med, flags, 13, px, py, sm, emission_scale=2.5, density=dv)
    want = ref.render_ext_paths(s.camera, med, 13, px, py, sm, flags, emission_scale=2.5, density=vol)
    L = got["L"].cpu().numpy().astype(np.float64)
    Lo = want["L"]
    close = np.abs(L - Lo) <= REL * np.maximum(np.abs(Lo), 1e-6)
    assert close.mean() >= FRAC, (close.mean(), np.max(np.abs(L - Lo)))
    assert np.mean(got["collisions"].cpu().numpy() == want["collisions"]) >= FRAC
    d = L - Lo
    if d.std() > 0:
        assert abs(d.mean()) <= 3 * d.std() / math.sqrt(len(d)) + 1e-7
    assert (Lo > 0).mean() > 0.5


def test_extended_frame_is_the_sum_of_its_paths(small):
    import paper_2506_11510_gb300 as tv
    s, vol, grid, _ = small
    dv = torch.from_numpy(vol).cuda()
    flags = VOXEL | EMISSION | ALBEDO | GCHAN
    stats = tv.new_stats()
    img, _ = tv.tet_render_ext(grid, s.camera, s.medium, flags, 3, 17, emission_scale=1.5, density=dv, stats=stats)
    px, py, sm = all_paths(s.camera, 3)
    got = tv.tet_trace_ext_paths(grid, s.camera, s.medium, flags, 17, px, py, sm, emission_scale=1.5, density=dv)
    pix = py.astype(np.int64) * s.camera.width + px
    want = np.bincount(pix, weights=got["L"].double().cpu().numpy(), minlength=s.camera.width * s.camera.height)
    g = img.cpu().numpy().ravel().astype(np.float64)
    # the frame ends ratio tracking below 2^-80; trace mode walks every shadow ray to the boundary
    close = np.abs(g - want) <= 1e-4 * np.maximum(np.abs(want), 1e-4)
    assert close.mean() >= 0.999
    assert tv.stats_dict(stats)["paths"] == len(px)


def test_furnace_with_unit_albedo_in_the_voxel_medium(small):
    import paper_2506_11510_gb300 as tv
    s, vol, _, _ = small
    dv = torch.from_numpy(vol).cuda()
    grid = tv.build_scene_grid(s, dv)
    t, _, g = W.make_channels(s)
    grid.channels(dv, t.cuda(), torch.ones_like(dv), g.cuda())
    med = W.Medium(0.2, 0.0, 64.0, 100000, s.medium.sun_dir, 0.0, 1.0)
    px, py, sm = all_paths(s.camera, 1)
    r = tv.tet_trace_ext_paths(grid, s.camera, med, VOXEL | ALBEDO | GCHAN, 3, px, py, sm, density=dv)
    ok = (r["flags"].cpu().numpy() & 2) == 0
    assert ok.mean() > 0.999
    assert np.all(r["L"].cpu().numpy()[ok] == 1.0)


def test_voxel_medium_matches_the_regular_grid_comparator(small):
    """Delta tracking through the tet majorants and the DDA through the voxels
    render the same medium: frame means agree within 4 sigma."""
    import paper_2506_11510_gb300 as tv
    s, vol, grid, _ = small
    dv = torch.from_numpy(vol).cuda()
    spp = 256
    a, a2 = tv.tet_render_ext(grid, s.camera, s.medium, VOXEL, spp, 31, density=dv)
    b, b2 = tv.grid_render(dv, s.box_min, s.voxel_size, s.camera, s.medium, spp, 32)
    n = spp * a.numel()
    ma, mb = float(a.sum()) / n, float(b.sum()) / n
    va = float(a2.sum()) / n - ma * ma
    vb = float(b2.sum()) / n - mb * mb
    z = (ma - mb) / math.sqrt(va / n + vb / n)
    assert abs(z) < 4, z
