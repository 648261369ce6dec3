"""GPU LEB build (Sec. 2) against the CPU oracle: bit-exact codes, vertices,
tags, neighbour links, orientation ids, plane offsets, statistics, stored
densities and majorants."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2506_11510_gb300 import workloads as W
from tests import _checks as CK
from tests.conftest import scene_volume

pytestmark = pytest.mark.gpu

FIELDS = ("codes", "verts", "tag", "nbr", "nid", "plane", "density", "majorant", "count", "sum", "qmin", "qmax")


def gpu_arrays(grid):
    ex = grid.export()
    out = {k: v.cpu().numpy() for k, v in ex.items()}
    out["codes"] = out["codes"].view(np.uint64)
    out["sum"] = out["sum"].view(np.uint64)
    for k in ("count", "qmin", "qmax"):
        out[k] = out[k].view(np.uint32)
    return out


def assert_same_grid(gpu, ref):
    assert len(gpu["codes"]) == len(ref.codes), "tet counts differ: %d vs %d" % (len(gpu["codes"]), len(ref.codes))
    for k in FIELDS:
        g, r = gpu[k], getattr(ref, k)
        assert np.array_equal(g, r), "field %s differs at %d cells" % (k, int(np.sum(g != r)))


def build_both(s, vol):
    import paper_2506_11510_gb300 as tv
    grid = tv.build_scene_grid(s, torch.from_numpy(vol).cuda())
    ref = O.Grid.for_scene(s, vol).export()
    return grid, ref


@pytest.mark.parametrize("name", ["tiny", "adaptive_small", "production_small"])
def test_build_matches_oracle(name):
    s = W.scene(name)
    grid, ref = build_both(s, scene_volume(name))
    assert_same_grid(gpu_arrays(grid), ref)
    assert grid.info.K == ref.K and grid.info.max_depth == ref.max_depth and grid.info.rounds == ref.rounds


@pytest.mark.parametrize("fmt", [1, 2])
def test_build_density_formats(fmt):
    s = W.scene("adaptive_small", density_format=fmt)
    grid, ref = build_both(s, scene_volume("adaptive_small"))
    assert_same_grid(gpu_arrays(grid), ref)


@pytest.mark.parametrize("case", ["empty", "ragged_cubes", "uniform_d0", "uniform_d7", "no_camera", "camera_inside"])
def test_build_edge_cases(case):
    import paper_2506_11510_gb300 as tv
    base = W.scene("adaptive_small")
    rng = np.random.default_rng(5)
    if case == "empty":
        vol = np.zeros((16, 16, 16), np.float32)
        s = W.scene("adaptive_small", dims=(16, 16, 16), voxel_size=1 / 16, max_depth=12)
    elif case == "ragged_cubes":
        # 24 x 16 x 8 voxels: 3 x 2 x 1 cubes of 8^3, 36 roots
        vol = rng.uniform(0, 1, (8, 16, 24)).astype(np.float32)
        vol[vol < 0.4] = 0
        s = W.scene("adaptive_small", dims=(24, 16, 8), voxel_size=1 / 8, max_depth=12,
                    camera=W.Camera((1.5, 1.0, -2.5), (1.5, 1.0, 0.5), (0, 1, 0), 50.0, 40, 30))
    elif case == "uniform_d0":
        vol = scene_volume("tiny")
        s = W.scene("tiny", max_depth=0)
    elif case == "uniform_d7":
        vol = scene_volume("tiny")
        s = W.scene("tiny", max_depth=7)
    elif case == "no_camera":
        vol = scene_volume("adaptive_small")
        s = W.scene("adaptive_small", footprint_px=0.0, max_depth=12)
    else:
        vol = scene_volume("adaptive_small")
        s = W.with_camera(W.scene("adaptive_small", max_depth=15), pos=(0.4, 0.45, 0.5), target=(0.9, 0.5, 0.6))
    grid = tv.build_scene_grid(s, torch.from_numpy(np.ascontiguousarray(vol)).cuda())
    ref = O.Grid.for_scene(s, vol).export()
    assert_same_grid(gpu_arrays(grid), ref)
    CK.check_grid(ref)


def test_build_rejects_bad_arguments():
    import paper_2506_11510_gb300 as tv
    vol = torch.zeros((16, 16, 16), device="cuda")
    with pytest.raises(tv.TetvolError):
        tv.leb_build(vol, (0, 0, 0), 1 / 16, max_depth=51)
    with pytest.raises(tv.TetvolError):
        # 9 x 8 x 8 cubes of 2^3 voxels -> 3456 roots, more than the code's 8 root bits
        tv.leb_build(torch.zeros((16, 16, 18), device="cuda"), (0, 0, 0), 1 / 16, max_depth=3)
