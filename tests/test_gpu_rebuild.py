"""Rebuilds for a moved camera (leb_rebuild): reusing a previous grid's node
statistics must give exactly the grid a fresh build gives (and so the oracle's),
for small moves, large moves, a chain of rebuilds and changed build settings."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2506_11510_gb300 import workloads as W
from tests.conftest import scene_volume

pytestmark = pytest.mark.gpu

FIELDS = ("codes", "verts", "tag", "nbr", "nid", "plane", "density", "majorant", "count", "sum", "qmin", "qmax")


def _same(a, b):
    ea, eb = a.export(FIELDS), b.export(FIELDS)
    for k in FIELDS:
        assert torch.equal(ea[k], eb[k]), k


def _moved(s, dx=0.0, dy=0.0, dz=0.0, fov=None):
    c = s.camera
    pos = (c.pos[0] + dx, c.pos[1] + dy, c.pos[2] + dz)
    return W.with_camera(s, pos=pos, fov_y_deg=fov or c.fov_y_deg)


@pytest.mark.parametrize("name", ["adaptive_small", "production_small"])
def test_rebuild_equals_fresh_build(name):
    import paper_2506_11510_gb300 as tv
    s = W.scene(name)
    vol = torch.from_numpy(scene_volume(name)).cuda()
    g0 = tv.build_scene_grid(s, vol)
    for s1 in (_moved(s, dx=0.05), _moved(s, dx=-0.3, dz=0.4, fov=30.0), s):
        g1 = tv.rebuild_scene_grid(g0, s1, vol)
        _same(g1, tv.build_scene_grid(s1, vol))
    # the oracle's grid for the moved camera, bit for bit
    s1 = _moved(s, dx=-0.3, dz=0.4, fov=30.0)
    g1 = tv.rebuild_scene_grid(g0, s1, vol)
    ref = O.Grid.for_scene(s1, scene_volume(name)).export()
    ex = g1.export(("codes", "nbr", "density"))
    assert np.array_equal(ex["codes"].cpu().numpy().view(np.uint64), ref.codes)
    assert np.array_equal(ex["nbr"].cpu().numpy(), ref.nbr)
    assert np.array_equal(ex["density"].cpu().numpy(), ref.density)


def test_chain_of_rebuilds_and_changed_settings():
    import dataclasses
    import paper_2506_11510_gb300 as tv
    s = W.scene("adaptive_small")
    vol = torch.from_numpy(scene_volume("adaptive_small")).cuda()
    g = tv.build_scene_grid(s, vol)
    for k in range(4):
        sk = _moved(s, dx=0.04 * k, dy=-0.02 * k)
        g = tv.rebuild_scene_grid(g, sk, vol)
        _same(g, tv.build_scene_grid(sk, vol))
    s2 = dataclasses.replace(s, variation_threshold=0.3, footprint_px=2.0)
    _same(tv.rebuild_scene_grid(g, s2, vol), tv.build_scene_grid(s2, vol))


def test_rebuild_rejects_another_volume_shape():
    import paper_2506_11510_gb300 as tv
    from paper_2506_11510_gb300 import TetvolError
    s = W.scene("adaptive_small")
    vol = torch.from_numpy(scene_volume("adaptive_small")).cuda()
    g = tv.build_scene_grid(s, vol)
    other = torch.zeros((32, 64, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(TetvolError):
        tv.leb_rebuild(g, other, s.box_min, s.voxel_size, s.camera, s.footprint_px, s.variation_threshold,
                       s.max_depth, s.density_format)
